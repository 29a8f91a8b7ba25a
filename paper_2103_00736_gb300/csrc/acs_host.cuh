// Host-side preparation of one conic program, shared by the single-problem
// API (acs_capi.cu) and the batched API (acs_batch.cu): input validation,
// the relabelling of the constraints, the transpose, and the host image of
// the sliced-ELLPACK layout of A and A' (layout in acs_internal.cuh).
// Not part of the public ABI.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <exception>
#include <memory>
#include <new>
#include <system_error>
#include <thread>
#include <vector>

#include "../../include/acs.h"

namespace acs {
namespace host {

constexpr int kSortWindow = 2048;   // rows of A are sorted by length within windows of this size

// Host threads for preparing a matrix of `entries` stored entries: one below
// 2^20 entries (thread start-up would cost more than it saves, e.g. for each
// member of a batch), else one per hardware thread, at most 16.
inline int host_threads(long long entries) {
    if (entries < (1LL << 20)) return 1;
    const unsigned h = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(h, 16u));
}

// Runs f(0), ..., f(T-1) on up to T host threads (the caller runs f(0)); a
// part whose thread cannot be started runs on the caller afterwards.  Every
// part writes its own outputs, so the result does not depend on T or on
// the order in which the parts run.  An exception of a part (an allocation
// that failed) is rethrown on the caller once every part has ended.
template <typename F>
void parallel_for(int T, const F& f) {
    std::vector<std::exception_ptr> err((size_t)std::max(T, 1));
    auto run = [&f, &err](int t) {
        try {
            f(t);
        } catch (...) {
            err[t] = std::current_exception();
        }
    };
    std::vector<std::thread> th;
    std::vector<int> on_caller;
    for (int t = 1; t < T; ++t) {
        try {
            th.emplace_back(run, t);
        } catch (const std::system_error&) {
            on_caller.push_back(t);
        }
    }
    run(0);
    for (int t : on_caller) run(t);
    for (auto& x : th) x.join();
    for (auto& e : err)
        if (e) std::rethrow_exception(e);
}

// The C entry points call host code that allocates; a host allocation that
// fails (the only exception this code raises) must not leave through the C
// ABI as an exception: it becomes ACS_ERR_OOM.
template <typename F>
int no_throw(const F& f) {
    try {
        return f();
    } catch (...) {
        return ACS_ERR_OOM;
    }
}

// [lo, hi) of part t of T equal parts of [0, N).
inline long long part_lo(long long N, int t, int T) { return N * t / T; }

// Vectors whose resize leaves the new elements uninitialised: the large host
// images are written in full by the threads that fill them, so their pages
// are first touched (and zeroed by the OS) in parallel, not by one thread.
template <typename T>
struct uninit_alloc : std::allocator<T> {
    template <typename U>
    struct rebind { using other = uninit_alloc<U>; };
    uninit_alloc() = default;
    template <typename U>
    uninit_alloc(const uninit_alloc<U>&) {}
    template <typename U>
    void construct(U* p) noexcept { ::new ((void*)p) U; }
    template <typename U, typename... A>
    void construct(U* p, A&&... a) { ::new ((void*)p) U(std::forward<A>(a)...); }
};
template <typename T>
using raw_vector = std::vector<T, uninit_alloc<T>>;

inline bool finite_all(const double* v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// Checks of the problem statement (Section II, Eq. (1)) as the ABI states
// them: CSR shape and order, finite data, cone sizes adding up to n.
inline int validate(int32_t m, int32_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                    const double* b, const double* c, int32_t n_orthant, int32_t n_soc,
                    const int32_t* soc_dims) {
    if (m <= 0 || n <= 0 || !row_ptr || !b || !c) return ACS_ERR_ARG;
    if (row_ptr[0] != 0) return ACS_ERR_CSR;
    for (int i = 0; i < m; ++i)
        if (row_ptr[i + 1] <= row_ptr[i]) return ACS_ERR_CSR;    // non-monotone or empty row
    const int64_t nnz64 = row_ptr[m];
    if (nnz64 <= 0 || nnz64 >= (int64_t)1 << 31) return ACS_ERR_CSR;
    if (!col || !val) return ACS_ERR_ARG;
    const int nnz = (int)nnz64;
    // the per-entry checks run over row ranges in parallel; each kind of
    // check is decided over all rows before the next, so the code returned
    // is the one a single pass in this order would return
    const int T = host_threads(nnz);
    std::vector<char> bad_col(T, 0), bad_val(T, 0);
    parallel_for(T, [&](int t) {
        const int i1 = (int)part_lo(m, t + 1, T);
        for (int i = (int)part_lo(m, t, T); i < i1 && !bad_col[t]; ++i) {
            int prev = -1;
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                const int j = col[k];
                if (j < 0 || j >= n || j <= prev) { bad_col[t] = 1; break; }
                prev = j;
            }
        }
        const long long k0 = part_lo(nnz, t, T), k1 = part_lo(nnz, t + 1, T);
        bad_val[t] = finite_all(val + k0, (size_t)(k1 - k0)) ? 0 : 1;
    });
    for (char f : bad_col)
        if (f) return ACS_ERR_CSR;
    for (char f : bad_val)
        if (f) return ACS_ERR_ARG;
    if (!finite_all(b, m) || !finite_all(c, n)) return ACS_ERR_ARG;
    if (n_orthant < 0 || n_soc < 0 || (n_soc > 0 && !soc_dims)) return ACS_ERR_CONES;
    int64_t tot = n_orthant;
    for (int i = 0; i < n_soc; ++i) {
        if (soc_dims[i] < 2) return ACS_ERR_CONES;
        tot += soc_dims[i];
    }
    if (tot != n) return ACS_ERR_CONES;
    return ACS_SOLVED;
}

constexpr int kDenseLimit = 4096;   // largest m for the cached dense projection operator
constexpr int kDenseRowsLimit = 16384;   // ... when every row of A is full (tiled assembly of M)

// Settings checks shared by every entry point that takes acs_settings.
inline bool valid_settings(const acs_settings& set) {
    return set.mu > 0 && set.t > 0 && set.check_every > 0 && set.cg_max_iter > 0 && set.cg_refine > 0 &&
           set.cg_refine <= 8 && set.cg_tol >= 0 && set.cg_eta >= 0 && set.cond_period >= 0 && set.cond_first >= 0 &&
           set.n_cond_list >= 0 && !(set.n_cond_list > 0 && !set.cond_list) &&
           (set.precision == ACS_PREC_MIXED || set.precision == ACS_PREC_FP32 ||
            set.precision == ACS_PREC_FP64) &&
           set.col_block >= -1 && set.outer32_tol >= 0 && set.polish_tol >= 0 &&
           (set.splitting == ACS_SPLIT_DR ||
            (set.splitting == ACS_SPLIT_ADMM && set.cond_first == 0 && set.n_cond_list == 0)) &&
           (set.projection == ACS_PROJ_AUTO || set.projection == ACS_PROJ_CG || set.projection == ACS_PROJ_DENSE) &&
           set.dense_max_m >= 0 && set.dense_max_m <= kDenseLimit && set.dense_switch_max_m >= 0 &&
           set.dense_switch_max_m <= kDenseLimit && set.dense_switch_cg >= 0 &&
           (set.a_storage == ACS_STORE_FP32 || set.a_storage == ACS_STORE_BF16) &&
           set.extrapolation >= 0 && set.extrapolation <= 2;
}

// BF16 bit pattern of a finite value: the upper 16 bits of its FP32 value,
// rounded to nearest with ties to even.
inline unsigned short to_bf16(double v) {
    const float f = (float)v;
    unsigned u;
    memcpy(&u, &f, sizeof(u));
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (unsigned short)(u >> 16);
}

// CG iterations after a rescaling that cost about one factorisation of the
// cached operator ((2/3) m^3 FP64 flops against 2 sparse passes over nnz
// stored entries per CG iteration; the factor 0.3 is measured on this GPU:
// one factorisation of an m = 1000, 5e4-nonzero M costs ~5700 CG iterations),
// and at least 8 * dense_switch_cg.  Full rows (nnz = m n): the tiled
// assembly adds m^2 n / 2 multiply-adds, and the factor is 1.0 instead,
// m^2 / n CG iterations (measured: one factorisation takes 109 ms at m = 2320,
// n = 2900 against 60 us a CG iteration, 1.73 s at m = 8000, n = 1e4 against
// 0.35 ms).
inline long long switch_budget(const acs_settings& set, int m, long long nnz, bool full_rows = false) {
    const double k = full_rows ? 1.0 : 0.3;
    const double f = k * (double)m * (double)m * (double)m / (double)(nnz > 0 ? nnz : 1);
    return std::max((long long)8 * set.dense_switch_cg, (long long)f);
}

// How a problem with m constraints applies the projection: 0 = CG only,
// 1 = the cached dense operator from the first iteration, 2 = CG, switching
// to the cached operator if CG stalls.
inline int dense_mode(const acs_settings& set, int m, bool full_rows = false) {
    if (set.projection == ACS_PROJ_DENSE) return m <= (full_rows ? kDenseRowsLimit : kDenseLimit) ? 1 : 0;
    if (set.projection != ACS_PROJ_AUTO) return 0;
    // full rows (the dense workloads): M costs m^2 n / 2 + 2 m^3 / 3 FP64 multiply-adds at a
    // rescaling (the tiled assembly, the factor, its inverse) against ~2 m n a CG iteration; the
    // switch budget 0.3 m^3 / nnz = 0.3 m^2 / n CG iterations matches that ratio on this GPU, so
    // the rule of the sparse case decides: the dense LPs (t = 9.2), whose rescaled M stalls
    // Jacobi-CG, switch; the dense SOCPs (t = 1.7) mostly stay on CG
    if (full_rows && m <= kDenseRowsLimit && m > set.dense_switch_max_m) return 2;
    if (m <= set.dense_max_m) return 1;
    if (set.dense_switch_cg > 0 && m <= set.dense_switch_max_m) return 2;
    return 0;
}


// Host image of a sliced-ELLPACK matrix with G lanes per row.
struct HostSell {
    int nrows = 0, nslices = 0, g = 1;
    std::vector<int> sptr, slen;
    raw_vector<int> col;
    raw_vector<double> val;
};

// Rows are given by (beg[r], end[r]) ranges into (cols, vals); padding
// entries repeat column 0 with value 0.  nslices = -1 if the padded size
// does not fit 32-bit offsets.
// Slice table of a sliced-ELLPACK image with g lanes per row for rows of the
// given lengths (len(r), r < nrows): chunks per slice (slen) and the start
// of each slice (sptr, nslices + 1 entries); returns the image's size in
// entries (>= INT32_MAX: does not fit 32-bit offsets).
template <typename Len>
long long sell_shape(int nrows, int g, const Len& len, std::vector<int>& sptr, std::vector<int>& slen) {
    const int h = 32 / g;                     // rows per slice
    const int nslices = (nrows + h - 1) / h;
    sptr.assign(nslices + 1, 0);
    slen.assign(nslices, 0);
    long long total = 0;
    for (int sl = 0; sl < nslices; ++sl) {
        long long mx = 0;
        for (int r = sl * h; r < std::min(nrows, sl * h + h); ++r) mx = std::max<long long>(mx, len(r));
        const long long chunks = (mx + g - 1) / g;
        slen[sl] = (int)chunks;
        sptr[sl] = (int)std::min<long long>(total, INT32_MAX);
        total += 32 * chunks;
    }
    sptr[nslices] = (int)std::min<long long>(total, INT32_MAX);
    return total;
}

inline HostSell build_sell(int nrows, int g, const std::vector<long long>& beg, const std::vector<long long>& end,
                           const int* cols, const double* vals, int threads = 1) {
    HostSell H;
    const int h = 32 / g;                     // rows per slice
    H.nrows = nrows;
    H.g = g;
    H.nslices = (nrows + h - 1) / h;
    const long long total = sell_shape(nrows, g, [&](int r) { return end[r] - beg[r]; }, H.sptr, H.slen);
    if (total >= INT32_MAX) { H.col.clear(); H.nslices = -1; return H; }
    H.col.resize(total);
    H.val.resize(total);
    // slices own disjoint ranges of the image: zero (the padding) and fill
    // them in parallel
    parallel_for(threads, [&](int t) {
        const int s0 = (int)part_lo(H.nslices, t, threads), s1 = (int)part_lo(H.nslices, t + 1, threads);
        std::fill(H.col.begin() + H.sptr[s0], H.col.begin() + H.sptr[s1], 0);
        std::fill(H.val.begin() + H.sptr[s0], H.val.begin() + H.sptr[s1], 0.0);
        for (int sl = s0; sl < s1; ++sl)
            for (int lr = 0; lr < h; ++lr) {
                const int r = sl * h + lr;
                if (r >= nrows) break;
                long long k = 0;
                for (long long e = beg[r]; e < end[r]; ++e, ++k) {
                    const long long idx = H.sptr[sl] + 32 * (k / g) + lr * g + (k % g);
                    H.col[idx] = cols[e];
                    H.val[idx] = vals[e];
                }
            }
    });
    return H;
}

// Lanes per row: enough slices for four per warp of the team that runs the
// products (load balance), but no more lanes than the average row length.
inline int choose_g(long long nrows, long long nnz, long long warps) {
    const double avg = nrows > 0 ? (double)nnz / (double)nrows : 1.0;
    int g = 1;
    while (g < 32 && (nrows * g) / 32 < 4 * warps && 2 * g <= avg) g *= 2;
    return g;
}

// A' of the relabelled A: for each coordinate j, the relabelled rows r with
// A[perm[r], j] != 0, in increasing order, as CSR (rpT[n + 1], rows, vals).
// Below 2^20 entries a plain counting sort (one pass, everything in cache).
// Above, a counting sort would scatter every entry to a random place in
// arrays of 12 bytes per entry; instead the entries first go to buckets of
// kBucketCols consecutive columns (pass 2), then each bucket is sorted by
// column within a cache-sized window (pass 3).  Thread t takes the relabelled rows
// [m t / T, m (t + 1) / T) in passes 1 and 2 and places its entries after
// those of the threads before it in every bucket, so every bucket holds its
// entries in increasing row order and the stable sort of pass 3 keeps it:
// the result is the same for any number of threads.
constexpr int kBucketCols = 1024;

inline void transpose_relabelled(int m, int n, const int64_t* row_ptr, const int32_t* col, const double* val,
                                 const std::vector<int>& perm, int T, std::vector<long long>& rpT,
                                 raw_vector<int>& rows, raw_vector<double>& vals) {
    const long long nnz = row_ptr[m];
    if (nnz < (1LL << 20)) {
        rpT.assign((size_t)n + 1, 0);
        for (long long k = 0; k < nnz; ++k) rpT[col[k] + 1]++;
        for (int j = 0; j < n; ++j) rpT[j + 1] += rpT[j];
        rows.resize(nnz);
        vals.resize(nnz);
        std::vector<long long> cur(rpT.begin(), rpT.end() - 1);
        for (int r = 0; r < m; ++r) {
            const int i = perm[r];
            for (long long k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                const long long d = cur[col[k]]++;
                rows[d] = r;
                vals[d] = val[k];
            }
        }
        return;
    }
    const int B = (n + kBucketCols - 1) / kBucketCols;
    // pass 1: entries per (thread, bucket)
    std::vector<long long> cnt((size_t)T * B, 0);
    parallel_for(T, [&](int t) {
        long long* c = cnt.data() + (size_t)t * B;
        const int r1 = (int)part_lo(m, t + 1, T);
        for (int r = (int)part_lo(m, t, T); r < r1; ++r) {
            const int i = perm[r];
            for (long long k = row_ptr[i]; k < row_ptr[i + 1]; ++k) ++c[col[k] / kBucketCols];
        }
    });
    // bucket by bucket, thread by thread: where each thread's entries go
    std::vector<long long> off((size_t)T * B), bstart((size_t)B + 1);
    long long pos = 0;
    for (int b = 0; b < B; ++b) {
        bstart[b] = pos;
        for (int t = 0; t < T; ++t) {
            off[(size_t)t * B + b] = pos;
            pos += cnt[(size_t)t * B + b];
        }
    }
    bstart[B] = pos;
    // pass 2: stage (row, column, value) in the buckets
    raw_vector<int> sr(nnz), sc(nnz);
    raw_vector<double> sv(nnz);
    parallel_for(T, [&](int t) {
        long long* o = off.data() + (size_t)t * B;
        const int r1 = (int)part_lo(m, t + 1, T);
        for (int r = (int)part_lo(m, t, T); r < r1; ++r) {
            const int i = perm[r];
            for (long long k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                const long long p = o[col[k] / kBucketCols]++;
                sr[p] = r;
                sc[p] = col[k];
                sv[p] = val[k];
            }
        }
    });
    // pass 3: a stable counting sort by column inside every bucket
    rpT.assign((size_t)n + 1, 0);
    rows.resize(nnz);
    vals.resize(nnz);
    parallel_for(T, [&](int t) {
        std::vector<long long> cur(kBucketCols + 1);
        const int b1 = (int)part_lo(B, t + 1, T);
        for (int b = (int)part_lo(B, t, T); b < b1; ++b) {
            const int j0 = b * kBucketCols, w = std::min(n, j0 + kBucketCols) - j0;
            std::fill(cur.begin(), cur.begin() + w + 1, 0LL);
            for (long long p = bstart[b]; p < bstart[b + 1]; ++p) ++cur[sc[p] - j0 + 1];
            cur[0] = bstart[b];
            for (int q = 0; q < w; ++q) cur[q + 1] += cur[q];
            for (int q = 0; q < w; ++q) rpT[j0 + q] = cur[q];
            for (long long p = bstart[b]; p < bstart[b + 1]; ++p) {
                const long long d = cur[sc[p] - j0]++;
                rows[d] = sr[p];
                vals[d] = sv[p];
            }
        }
    });
    rpT[n] = nnz;
}

// Everything the device needs of one problem, in host memory.  Row r of the
// device matrix is row perm[r] of the caller's A (b, y and w live in that
// order); A' lists, for each coordinate, the relabelled rows touching it in
// increasing order.
struct HostProblem {
    std::vector<int> perm;
    HostSell A, AT;
    std::vector<double> bperm;
    std::vector<int> soc_off;      // n_soc + 1 absolute offsets
    double bnorm = 0, cnorm = 0;
};

// warps_A / warps_AT: warps of the team that will run the products over the
// rows of A and of A' (sets the lanes per row).  Inputs must have passed
// validate().  Returns ACS_ERR_CSR if a padded matrix exceeds 32-bit offsets.
// The transpose of the relabelled A as CSR (built on the way; kept for a
// caller that builds another image of A' from it).
struct HostTranspose {
    std::vector<long long> rp;
    raw_vector<int> rows;
    raw_vector<double> vals;
};

// Everything of the host preparation but the matrix images: the relabelling
// (rows sorted by length, descending, within windows, so that the rows of a
// slice have similar lengths and padding is small), b in that order, the cone
// offsets and the norms of b and c.
inline void build_meta(int32_t m, int32_t n, const int64_t* row_ptr, const double* b, const double* c,
                       int32_t n_orthant, int32_t n_soc, const int32_t* soc_dims, HostProblem& H) {
    const long long nnz = row_ptr[m];
    std::vector<int>& perm = H.perm;
    perm.resize(m);
    const int T = host_threads(nnz);
    const int nwin = (m + kSortWindow - 1) / kSortWindow;
    const int tt = std::min(T, nwin);
    parallel_for(tt, [&](int t) {                            // windows are independent
        for (int w = (int)part_lo(nwin, t, tt); w < (int)part_lo(nwin, t + 1, tt); ++w) {
            const int w0 = w * kSortWindow, w1 = std::min(m, w0 + kSortWindow);
            for (int i = w0; i < w1; ++i) perm[i] = i;
            std::stable_sort(perm.begin() + w0, perm.begin() + w1, [&](int a, int b2) {
                return (row_ptr[a + 1] - row_ptr[a]) > (row_ptr[b2 + 1] - row_ptr[b2]);
            });
        }
    });
    H.bperm.resize(m);
    for (int r = 0; r < m; ++r) H.bperm[r] = b[perm[r]];
    H.soc_off.resize(n_soc + 1);
    H.soc_off[0] = n_orthant;
    for (int i = 0; i < n_soc; ++i) H.soc_off[i + 1] = H.soc_off[i] + soc_dims[i];
    double bn = 0, cn = 0;
    for (int i = 0; i < m; ++i) bn += b[i] * b[i];
    for (int j = 0; j < n; ++j) cn += c[j] * c[j];
    H.bnorm = sqrt(bn);
    H.cnorm = sqrt(cn);
}

inline int build(int32_t m, int32_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                 const double* b, const double* c, int32_t n_orthant, int32_t n_soc, const int32_t* soc_dims,
                 long long warps_A, long long warps_AT, HostProblem& H, HostTranspose* keep_T = nullptr) {
    const int nnz = (int)row_ptr[m];
    build_meta(m, n, row_ptr, b, c, n_orthant, n_soc, soc_dims, H);
    const std::vector<int>& perm = H.perm;
    const int T = host_threads(nnz);
    {
        std::vector<long long> beg(m), end(m);
        for (int r = 0; r < m; ++r) { beg[r] = row_ptr[perm[r]]; end[r] = row_ptr[perm[r] + 1]; }
        H.A = build_sell(m, choose_g(m, nnz, warps_A), beg, end, col, val, T);
    }
    {
        std::vector<long long> rpT;
        raw_vector<int> ciT;
        raw_vector<double> valT;
        transpose_relabelled(m, n, row_ptr, col, val, perm, T, rpT, ciT, valT);
        std::vector<long long> beg(rpT.begin(), rpT.end() - 1), end(rpT.begin() + 1, rpT.end());
        H.AT = build_sell(n, choose_g(n, nnz, warps_AT), beg, end, ciT.data(), valT.data(), T);
        if (keep_T) {
            keep_T->rp.swap(rpT);
            keep_T->rows.swap(ciT);
            keep_T->vals.swap(valT);
        }
    }
    if (H.A.nslices < 0 || H.AT.nslices < 0) return ACS_ERR_CSR;
    return ACS_SOLVED;
}

}  // namespace host
}  // namespace acs
