// Column-blocked sliced ELLPACK: the layout of the FP32 matrix passes of the
// single-problem launch.  Not part of the public ABI.
//
// A sliced-ELLPACK pass gathers one entry of the multiplied vector per
// nonzero.  For the random sparsity of the large LP and SOCP that vector
// (0.8 to 4 MB) lives in L2, and every gather is a separate L2 sector
// request: the passes run at the L2's random-request rate, far below the
// HBM bandwidth that streams the matrix.  Here the columns are cut into
// blocks of at most `width` columns (one block of FP32 vector entries fills
// a CTA's shared memory), and every block of columns is stored as its own
// sliced-ELLPACK matrix:
//
//   item = (block b, slice q): the entries of 32 rows that fall in block b;
//     lane r of the item holds row  (q / kCbSliceWin) * kCbWindow + rowid[item*32 + r]
//     (rows are sorted by their entry count in block b within windows of
//     kCbWindow rows, so that the rows of a slice have similar counts);
//     entry k of that row sits at  sptr[item] + 32 k + r;
//     col = column - b * width (16 bits), val = the FP32 value;
//     padding entries have col 0 and val 0; rowid 0xFFFF marks no row;
//     every item has at least one chunk, and bit c % 32 of cend[c / 32]
//     marks chunk c (in units of 32 entries) as the last of its item;
//     ipos[b * nsl * 32 + row] = the slot of the row within its window in
//     block b (the inverse of rowid).
//
// A pass stages block b of the vector in shared memory and multiplies every
// item of the block, writing one partial sum per row and block,
// part[b * nrows + row].  A later phase adds the partials of a row in block
// order, so the result depends only on the layout, not on the launch.  The
// items are dealt to the CTAs of the launch as contiguous ranges of equal
// work (cta_beg), block-major, so a CTA stages at most a few blocks.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

#include "acs_host.cuh"
#include "acs_internal.cuh"

namespace acs {

// Columns of one block: FP32 vector entries staged in shared memory.  The
// persistent kernel's static shared memory (reductions) leaves this much of
// the 227 KB a CTA may use.
constexpr int kCbMaxWidth = 49152;

namespace host {

struct HostCb {
    int nrows = 0, ncols = 0, width = 0, nblocks = 0, nsl = 0;
    std::vector<int> sptr;
    std::vector<unsigned short> rowid;
    raw_vector<unsigned short> col;
    raw_vector<float> val;
    std::vector<int> cta_beg;
    std::vector<unsigned> cend;
    std::vector<unsigned short> ipos;      // [nblocks * nsl * 32]: slot of each row in its window
};

// Block width for ncols columns and a limit: the fewest blocks that respect
// the limit, made as even as possible, rounded up to a multiple of 4 (each
// block then starts on a 16-byte boundary of an FP32 vector).
inline int cb_width(int ncols, int limit) {
    limit = std::max(4, limit - limit % 4);
    const long long nb = (ncols + (long long)limit - 1) / limit;
    long long w = (ncols + nb - 1) / nb;
    w = (w + 3) / 4 * 4;
    return (int)std::min<long long>(w, limit);
}

// Deals items [0, nitems) to `ctas` contiguous ranges of about equal work;
// the work of an item is its chunks plus one (slice bookkeeping).
inline std::vector<int> cb_deal(const std::vector<int>& sptr, int ctas) {
    const int nitems = (int)sptr.size() - 1;
    std::vector<int> beg((size_t)ctas + 1, nitems);
    long long total = 0;
    for (int it = 0; it < nitems; ++it) total += (sptr[it + 1] - sptr[it]) / 32 + 1;
    long long acc = 0;
    int c = 0;
    beg[0] = 0;
    for (int it = 0; it < nitems && c + 1 < ctas; ++it) {
        acc += (sptr[it + 1] - sptr[it]) / 32 + 1;
        while (c + 1 < ctas && acc * ctas >= total * (long long)(c + 1)) beg[++c] = it + 1;
    }
    for (int k = c + 1; k <= ctas; ++k) beg[k] = nitems;
    return beg;
}

// Rows given by (beg[r], end[r]) ranges into (cols, vals), columns strictly
// increasing within each row (true of the validated A and of its transpose).
// Returns false if the padded image exceeds 32-bit offsets.
inline bool build_cbsell(int nrows, int ncols, int width, const std::vector<long long>& beg,
                         const std::vector<long long>& end, const int* cols, const double* vals, int ctas,
                         int threads, HostCb& H) {
    H.nrows = nrows;
    H.ncols = ncols;
    H.width = width;
    H.nblocks = (ncols + width - 1) / width;
    H.nsl = (nrows + 31) / 32;
    const int nb = H.nblocks, R = nrows, nsl = H.nsl;
    const long long nitems = (long long)nb * nsl;
    // entries of every row in every block
    std::vector<int> cnt((size_t)nb * R, 0);
    parallel_for(threads, [&](int t) {
        const int r1 = (int)part_lo(R, t + 1, threads);
        for (int r = (int)part_lo(R, t, threads); r < r1; ++r)
            for (long long e = beg[r]; e < end[r]; ++e) ++cnt[(size_t)(cols[e] / width) * R + r];
    });
    // per block and window: rows by decreasing count (stable); pos = place in that order
    const int nwin = (R + kCbWindow - 1) / kCbWindow;
    std::vector<int> pos((size_t)nb * R);
    H.rowid.assign((size_t)nitems * 32, kCbNoRow);
    H.ipos.assign((size_t)nitems * 32, 0);
    std::vector<int> len((size_t)nitems, 0);
    parallel_for(threads, [&](int t) {
        std::vector<int> order;
        const long long u1 = part_lo((long long)nb * nwin, t + 1, threads);
        for (long long u = part_lo((long long)nb * nwin, t, threads); u < u1; ++u) {
            const int b = (int)(u / nwin), w = (int)(u % nwin);
            const int r0 = w * kCbWindow, r1 = std::min(R, r0 + kCbWindow);
            const int* cb = cnt.data() + (size_t)b * R;
            order.resize(r1 - r0);
            for (int k = 0; k < r1 - r0; ++k) order[k] = r0 + k;
            std::stable_sort(order.begin(), order.end(), [cb](int a, int c) { return cb[a] > cb[c]; });
            for (int k = 0; k < r1 - r0; ++k) {
                const int r = order[k];
                pos[(size_t)b * R + r] = k;
                H.ipos[(size_t)b * nsl * 32 + (size_t)r] = (unsigned short)k;
                const long long item = (long long)b * nsl + (long long)w * kCbSliceWin + k / 32;
                H.rowid[(size_t)item * 32 + (k % 32)] = (unsigned short)(r - r0);
                // the slice's longest row comes first; an item has at least
                // one chunk (a run of items is streamed chunk by chunk, and
                // every item's end is marked on a chunk)
                if (k % 32 == 0) len[(size_t)item] = std::max(1, cb[r]);
            }
        }
    });
    H.sptr.assign((size_t)nitems + 1, 0);
    long long total = 0;
    for (long long it = 0; it < nitems; ++it) {
        H.sptr[(size_t)it] = (int)std::min<long long>(total, INT32_MAX);
        total += 32LL * len[(size_t)it];
    }
    H.sptr[(size_t)nitems] = (int)std::min<long long>(total, INT32_MAX);
    if (total >= INT32_MAX) return false;
    H.col.resize((size_t)total);
    H.val.resize((size_t)total);
    // padding first (items own disjoint ranges), then the entries, row by row
    parallel_for(threads, [&](int t) {
        const long long i0 = part_lo(nitems, t, threads), i1 = part_lo(nitems, t + 1, threads);
        std::fill(H.col.begin() + H.sptr[(size_t)i0], H.col.begin() + H.sptr[(size_t)i1], (unsigned short)0);
        std::fill(H.val.begin() + H.sptr[(size_t)i0], H.val.begin() + H.sptr[(size_t)i1], 0.0f);
    });
    parallel_for(threads, [&](int t) {
        const int r1 = (int)part_lo(R, t + 1, threads);
        for (int r = (int)part_lo(R, t, threads); r < r1; ++r) {
            const int w = r / kCbWindow;
            int bcur = -1;
            long long k = 0, base = 0;
            for (long long e = beg[r]; e < end[r]; ++e) {
                const int j = cols[e];
                const int b = j / width;
                if (b != bcur) {                       // columns increase: a block's entries are contiguous
                    bcur = b;
                    k = 0;
                    const int p = pos[(size_t)b * R + r];
                    const long long item = (long long)b * nsl + (long long)w * kCbSliceWin + p / 32;
                    base = (long long)H.sptr[(size_t)item] + (p % 32);
                }
                const long long idx = base + 32 * k;
                H.col[(size_t)idx] = (unsigned short)(j - b * width);
                H.val[(size_t)idx] = (float)vals[e];
                ++k;
            }
        }
    });
    // end marks: bit c % 32 of word c / 32 is set if chunk c is the last
    // chunk of its item (one word more than needed, so that two consecutive
    // words can always be read)
    const long long nchunks = total / 32;
    H.cend.assign((size_t)(nchunks / 32 + 2), 0u);
    for (long long it = 0; it < nitems; ++it) {
        const long long last = (long long)H.sptr[(size_t)it + 1] / 32 - 1;
        H.cend[(size_t)(last / 32)] |= 1u << (last % 32);
    }
    H.cta_beg = cb_deal(H.sptr, ctas);
    return true;
}

}  // namespace host
}  // namespace acs
