// Sliced-ELLPACK images of A and A' built on the device from the caller's
// CSR (single-problem create): the same images the host builder makes
// (acs_host.cuh: build_sell, transpose_relabelled), bit for bit, with the
// host doing only the O(m) slice table of A; A''s column offsets and slice
// table are prefix sums on the device.
//
//   A : relabelled row r = row perm[r] of the CSR, entries in CSR order;
//       entry k of local row lr of slice sl at sptr[sl] + 32 (k / g) +
//       lr g + k % g; padding column 0, value 0.
//   A': row j = the relabelled rows r with A[perm[r], j] != 0, increasing:
//       entries counted per column, scattered (any order), then each column
//       sorted by r (the keys are distinct, so the result does not depend on
//       the scatter's order) and packed like A.
// Columns longer than kDevSortMax entries are left to the host builder.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <utility>
#include <vector>

#include "acs_host.cuh"
#include "acs_internal.cuh"

namespace acs {
namespace {

constexpr int kDevSortMax = 4096;         // longest column sorted in one CTA's shared memory
constexpr int kShortSort = 32;            // columns up to this length: insertion sort by one thread

// warp per row: row r's len[r] entries from (src_col, src_val)[beg[r] ...]
__global__ void pack_rows(int nrows, int g, const int* __restrict__ sptr, const long long* __restrict__ beg,
                          const int* __restrict__ len, const int* __restrict__ src_col,
                          const double* __restrict__ src_val, int* __restrict__ col, double* __restrict__ val) {
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const int h = 32 / g;
    for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows; r += nw) {
        const int sl = (int)(r / h), lr = (int)(r % h);
        const long long b0 = beg[r], base = sptr[sl];
        const int L = len[r];
        for (int k = lane; k < L; k += 32) {
            const long long idx = base + 32LL * (k / g) + (long long)lr * g + (k % g);
            col[idx] = src_col[b0 + k];
            val[idx] = src_val[b0 + k];
        }
    }
}

__global__ void count_cols(long long nnz, const int* __restrict__ col, int* __restrict__ cnt) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (long long)gridDim.x * blockDim.x)
        atomicAdd(cnt + col[k], 1);
}

// warp per relabelled row: its entries to their columns' segments
__global__ void scatter_cols(int m, const long long* __restrict__ beg, const int* __restrict__ len,
                             const int* __restrict__ col, const double* __restrict__ val,
                             const long long* __restrict__ rpT, int* __restrict__ cur, int* __restrict__ rowsT,
                             double* __restrict__ valsT) {
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < m; r += nw) {
        const long long b0 = beg[r];
        const int L = len[r];
        for (int k = lane; k < L; k += 32) {
            const int j = col[b0 + k];
            const long long pos = rpT[j] + atomicAdd(cur + j, 1);
            rowsT[pos] = (int)r;
            valsT[pos] = val[b0 + k];
        }
    }
}

// thread per column of at most kShortSort entries: insertion sort by row
__global__ void sort_short(int n, const long long* __restrict__ rpT, const int* __restrict__ cnt,
                           int* __restrict__ rowsT, double* __restrict__ valsT) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int L = cnt[j];
        if (L < 2 || L > kShortSort) continue;
        int* rk = rowsT + rpT[j];
        double* rv = valsT + rpT[j];
        for (int a = 1; a < L; ++a) {
            const int key = rk[a];
            const double v = rv[a];
            int p = a - 1;
            while (p >= 0 && rk[p] > key) {
                rk[p + 1] = rk[p];
                rv[p + 1] = rv[p];
                --p;
            }
            rk[p + 1] = key;
            rv[p + 1] = v;
        }
    }
}

// CTA per longer column (listed in cols): bitonic sort in shared memory,
// padded to a power of two with keys that sort last
__global__ void sort_long(const int* __restrict__ cols, const long long* __restrict__ rpT,
                          const int* __restrict__ cnt, int* __restrict__ rowsT, double* __restrict__ valsT) {
    __shared__ int key[kDevSortMax];
    __shared__ double v[kDevSortMax];
    const int j = cols[blockIdx.x];
    const int L = cnt[j];
    int N = 1;
    while (N < L) N <<= 1;
    int* rk = rowsT + rpT[j];
    double* rv = valsT + rpT[j];
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        key[i] = i < L ? rk[i] : 0x7FFFFFFF;
        v[i] = i < L ? rv[i] : 0.0;
    }
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1)
        for (int s = k >> 1; s > 0; s >>= 1) {
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const int p = i ^ s;
                if (p > i) {
                    const bool up = (i & k) == 0;
                    if ((key[i] > key[p]) == up) {
                        const int tk = key[i];
                        key[i] = key[p];
                        key[p] = tk;
                        const double tv = v[i];
                        v[i] = v[p];
                        v[p] = tv;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        rk[i] = key[i];
        rv[i] = v[i];
    }
}

// Per slice of A' (h = 32 / g columns): its chunk count ceil(max cnt / g);
// info[0] set if a column is longer than kDevSortMax, the columns longer than
// kShortSort appended to longc (in any order: each is sorted on its own)
// with info[1] their count.
__global__ void col_slices(int n, int g, const int* __restrict__ cnt, int* __restrict__ slen,
                           long long* __restrict__ info, int* __restrict__ longc) {
    const int h = 32 / g;
    const long long nsl = ((long long)n + h - 1) / h;
    for (long long sl = (long long)blockIdx.x * blockDim.x + threadIdx.x; sl < nsl;
         sl += (long long)gridDim.x * blockDim.x) {
        int mx = 0;
        const long long r1 = sl * h + h < n ? sl * h + h : n;
        for (long long r = sl * h; r < r1; ++r) {
            const int L = cnt[r];
            mx = L > mx ? L : mx;
            if (L > kDevSortMax) info[0] = 1;
            else if (L > kShortSort) longc[atomicAdd((unsigned long long*)(info + 1), 1ULL)] = (int)r;
        }
        slen[sl] = (mx + g - 1) / g;
    }
}

// Exclusive prefix sums on the device, in three launches: the sum of each
// tile of kScanTile entries, an exclusive scan of those sums by one CTA, and
// each tile's own scan offset by its tile's sum.  Entry i is f(i); out(i,
// exclusive, inclusive) receives the sums before and through entry i.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

struct ColCount {                 // entry j: the column's count
    const int* cnt;
    __device__ long long operator()(long long j) const { return cnt[j]; }
};
struct SliceWidth {               // entry sl: the slice's stored entries
    const int* slen;
    __device__ long long operator()(long long sl) const { return 32LL * slen[sl]; }
};
struct OffsetsOut {               // int64 offsets[0..N]
    long long* off;
    long long N;
    __device__ void operator()(long long i, long long ex, long long in) const {
        off[i] = ex;
        if (i == N - 1) off[N] = in;
    }
};
struct SlicePtrOut {              // int32 slice pointers[0..N], clamped as the host tables are
    int* sptr;
    long long N;
    __device__ void operator()(long long i, long long ex, long long in) const {
        sptr[i] = (int)(ex < INT32_MAX ? ex : INT32_MAX);
        if (i == N - 1) sptr[N] = (int)(in < INT32_MAX ? in : INT32_MAX);
    }
};

// exclusive scan of x over the CTA (kScanThreads threads); returns it and
// leaves the CTA's total in *total
__device__ long long cta_exclusive(long long x, long long* warp_s, long long* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_s[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const long long w = lane < kScanThreads / 32 ? warp_s[lane] : 0;
        long long wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kScanThreads / 32) warp_s[lane] = wi - w;
        if (lane == kScanThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    const long long ex = warp_s[wid] + inc - x;
    __syncthreads();                                  // warp_s free for the next call
    return ex;
}

template <typename F>
__global__ void __launch_bounds__(kScanThreads) tile_sums(long long N, F f, long long* __restrict__ sums) {
    __shared__ long long warp_s[kScanThreads / 32];
    __shared__ long long total;
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    long long s = 0;
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < N) s += f(base + k);
    cta_exclusive(s, warp_s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// one CTA: sums[0..nb) replaced by their exclusive scan, the grand total to *grand
__global__ void __launch_bounds__(kScanThreads) scan_tile_sums(long long nb, long long* __restrict__ sums,
                                                               long long* __restrict__ grand) {
    __shared__ long long warp_s[kScanThreads / 32];
    __shared__ long long total;
    long long carry = 0;
    for (long long c0 = 0; c0 < nb; c0 += kScanThreads) {
        const long long i = c0 + threadIdx.x;
        const long long v = i < nb ? sums[i] : 0;
        const long long ex = cta_exclusive(v, warp_s, &total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;                               // every thread reads the same total
        __syncthreads();
    }
    if (threadIdx.x == 0) *grand = carry;
}

template <typename F, typename Out>
__global__ void __launch_bounds__(kScanThreads) tile_apply(long long N, F f, const long long* __restrict__ offs,
                                                           Out out) {
    __shared__ long long warp_s[kScanThreads / 32];
    __shared__ long long total;
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    long long v[kScanItems];
    long long s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < N ? f(base + k) : 0;
        s += v[k];
    }
    long long run = offs[blockIdx.x] + cta_exclusive(s, warp_s, &total);
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < N) out(base + k, run, run + v[k]);
        run += v[k];
    }
}

template <typename F, typename Out>
void exclusive_scan(long long N, F f, Out out, long long* sums, long long* grand, cudaStream_t st) {
    const long long nb = (N + kScanTile - 1) / kScanTile;
    tile_sums<<<(unsigned)nb, kScanThreads, 0, st>>>(N, f, sums);
    scan_tile_sums<<<1, kScanThreads, 0, st>>>(nb, sums, grand);
    tile_apply<<<(unsigned)nb, kScanThreads, 0, st>>>(N, f, sums, out);
}

// scratch from the device cache, released on every return (after the
// stream that used it has been synchronised, or when nothing was launched)
struct Scratch {
    int device;
    cudaStream_t stream;
    std::vector<std::pair<void*, size_t>> p;
    Scratch(int d, cudaStream_t s) : device(d), stream(s) {}
    template <typename T>
    T* get(size_t count) {
        size_t got = 0;
        void* q = dev_alloc(device, std::max<size_t>(count, 1) * sizeof(T), &got);
        if (!q) return nullptr;
        p.emplace_back(q, got);
        return static_cast<T*>(q);
    }
    ~Scratch() {
        cudaStreamSynchronize(stream);               // nothing in flight still uses the blocks
        for (auto& a : p) dev_release(device, a.first, a.second);
    }
};

// ACS_TRACE_CREATE set: the host time of each part of the device build on
// stderr, the stream synchronised before each stamp (only then) so that
// the asynchronous work is counted in the part that issued it
struct BuildTrace {
    const bool on = getenv("ACS_TRACE_CREATE") != nullptr;
    cudaStream_t stream;
    std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
    explicit BuildTrace(cudaStream_t s) : stream(s) {}
    void operator()(const char* what) {
        if (!on) return;
        cudaStreamSynchronize(stream);
        const auto u = std::chrono::steady_clock::now();
        fprintf(stderr, "acs create:   %-24s %8.2f ms\n", what, std::chrono::duration<double, std::milli>(u - t).count());
        t = u;
    }
};

inline unsigned grid_for(long long work, int per_block) {
    return (unsigned)std::max<long long>(1, std::min<long long>((work + per_block - 1) / per_block, 152LL * 16));
}

// The support's indicator O_j = (x_j > z_j) (the crossover polish's B).
__global__ void support_indicator(int n, const double* __restrict__ x, const double* __restrict__ z,
                                  double* __restrict__ O) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        O[j] = x[j] > z[j] ? 1.0 : 0.0;
}

// Entries of each row of A kept in A_B (nonzero value, column in the support).
__global__ void count_support_entries(const SellMat A, const double* __restrict__ O, int* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int g = A.g, h = 32 / g;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long sl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < A.nslices; sl += nw) {
        const int len = A.slen[sl];
        long long idx = A.sptr[sl] + lane;
        int c = 0;
        for (int k = 0; k < len; ++k, idx += 32) c += (A.v64[idx] != 0.0 && O[A.col[idx]] != 0.0) ? 1 : 0;
        for (int o = g / 2; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        const long long row = sl * h + lane / g;
        if ((lane & (g - 1)) == 0 && row < A.nrows) cnt[row] = c;
    }
}

// A_B in the layout of A (same lanes per row, its own slice table): each
// row's kept entries in their order in A, placed by a prefix count over the
// row's lanes chunk by chunk.
__global__ void pack_support_entries(const SellMat A, const double* __restrict__ O, const int* __restrict__ sptrB,
                                     int* __restrict__ colB, double* __restrict__ valB, float* __restrict__ valB32) {
    const int lane = threadIdx.x & 31;
    const int g = A.g, h = 32 / g, lr = lane / g, t = lane % g;
    const unsigned gmask = g == 32 ? 0xffffffffu : ((1u << g) - 1u);
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long sl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < A.nslices; sl += nw) {
        const int len = A.slen[sl];
        long long idx = A.sptr[sl] + lane;
        const long long base = sptrB[sl];
        int run = 0;                                    // kept entries of this lane's row so far
        for (int k = 0; k < len; ++k, idx += 32) {
            const double v = A.v64[idx];
            const int j = A.col[idx];
            const bool keep = v != 0.0 && O[j] != 0.0;
            const unsigned bits = (__ballot_sync(0xffffffffu, keep) >> (lr * g)) & gmask;
            if (keep) {
                const int pos = run + __popc(bits & ((1u << t) - 1u));
                const long long out = base + 32LL * (pos / g) + (long long)lr * g + (pos % g);
                colB[out] = j;
                valB[out] = v;
                if (valB32) valB32[out] = A.v32[idx];
            }
            run += __popc(bits);
        }
        (void)h;
    }
}

}  // namespace

// A_B: the rows of A restricted to the columns of the support x > z of the
// problem's current iterate, built on the device into the polish's buffers
// (allocated at the first call, sized like A's image).  Sets X.O to the
// support's indicator.  out: the image (FP64 values only).
int support_rows(Problem* P, SellMat& out, bool with_f32) {
    const int m = P->m, n = P->n;
    const SellMat& A = P->A;
    cudaStream_t st = P->stream;
    if (!P->bcol) {
        const size_t pa = (size_t)std::max<long long>(P->padded_A, 1);
        if (!P->alloc(&P->bcol, pa) || !P->alloc(&P->bval, pa) || !P->alloc(&P->bsptr, (size_t)A.nslices + 1) ||
            !P->alloc(&P->bslen, (size_t)std::max(A.nslices, 1)) || !P->alloc(&P->bcnt, (size_t)m)) {
            P->bcol = nullptr;
            return ACS_ERR_OOM;
        }
    }
    if (with_f32 && !P->bval32 && !P->alloc(&P->bval32, (size_t)std::max<long long>(P->padded_A, 1)))
        return ACS_ERR_OOM;
    support_indicator<<<grid_for(n, 256), 256, 0, st>>>(n, P->x, P->z, P->X.O);
    count_support_entries<<<grid_for(32LL * A.nslices, 256), 256, 0, st>>>(A, P->X.O, P->bcnt);
    std::vector<int> cnt(m);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(cnt.data(), P->bcnt, sizeof(int) * m, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ACS_ERR_CUDA;
    std::vector<int> sptr, slen;
    const long long tot = host::sell_shape(m, A.g, [&](int r) { return (long long)cnt[r]; }, sptr, slen);
    if (tot > P->padded_A) return ACS_ERR_CSR;             // cannot happen: a subset of A's entries
    if (cudaMemcpyAsync(P->bsptr, sptr.data(), sizeof(int) * sptr.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(P->bslen, slen.data(), sizeof(int) * slen.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(P->bcol, 0, sizeof(int) * std::max<long long>(tot, 1), st) != cudaSuccess ||
        cudaMemsetAsync(P->bval, 0, sizeof(double) * std::max<long long>(tot, 1), st) != cudaSuccess)
        return ACS_ERR_CUDA;
    if (with_f32 && cudaMemsetAsync(P->bval32, 0, sizeof(float) * std::max<long long>(tot, 1), st) != cudaSuccess)
        return ACS_ERR_CUDA;
    pack_support_entries<<<grid_for(32LL * A.nslices, 256), 256, 0, st>>>(A, P->X.O, P->bsptr, P->bcol, P->bval,
                                                                          with_f32 ? P->bval32 : nullptr);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return ACS_ERR_CUDA;
    out = SellMat{};
    out.nrows = m;
    out.nslices = A.nslices;
    out.g = A.g;
    out.sptr = P->bsptr;
    out.slen = P->bslen;
    out.col = P->bcol;
    out.v64 = P->bval;
    out.v32 = with_f32 ? P->bval32 : nullptr;
    out.v16 = nullptr;
    P->padded_B = tot;
    return ACS_SOLVED;
}

int device_sell(Problem* P, const int64_t* row_ptr, const int32_t* col, const double* val,
                const std::vector<int>& perm, int gA, int gAT, DeviceSell& out) {
    const int m = P->m, n = P->n;
    const long long nnz = row_ptr[m];
    cudaStream_t st = P->stream;
    Scratch S(P->device, st);
    BuildTrace trace(st);
    // A: relabelled rows
    std::vector<long long> begA(m);
    std::vector<int> lenA(m);
    for (int r = 0; r < m; ++r) {
        begA[r] = row_ptr[perm[r]];
        lenA[r] = (int)(row_ptr[perm[r] + 1] - row_ptr[perm[r]]);
    }
    const long long totA = host::sell_shape(m, gA, [&](int r) { return (long long)lenA[r]; }, out.sptrA, out.slenA);
    if (totA >= INT32_MAX) return ACS_ERR_CSR;
    trace("tables of A");
    int* d_col = S.get<int>((size_t)nnz);
    double* d_val = S.get<double>((size_t)nnz);
    long long* d_begA = S.get<long long>(m);
    int* d_lenA = S.get<int>(m);
    int* d_cnt = S.get<int>(n);
    if (!d_col || !d_val || !d_begA || !d_lenA || !d_cnt) return ACS_ERR_OOM;
    trace("scratch");
    if (cudaMemcpyAsync(d_col, col, sizeof(int) * nnz, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_val, val, sizeof(double) * nnz, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_begA, begA.data(), sizeof(long long) * m, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_lenA, lenA.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(d_cnt, 0, sizeof(int) * n, st) != cudaSuccess)
        return ACS_ERR_CUDA;
    P->h2d_bytes += 12 * nnz + 12LL * m;
    trace("upload of the CSR");
    count_cols<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, d_col, d_cnt);
    // A': the slice table, the column offsets and the longer columns, on the
    // device; the host reads back the slice table and three counts
    const int hT = 32 / gAT;
    const long long nslT = ((long long)n + hT - 1) / hT;
    const long long nb = (std::max<long long>(n, nslT) + kScanTile - 1) / kScanTile;
    long long* d_rpT = S.get<long long>((size_t)n + 1);
    int* d_slT = S.get<int>((size_t)nslT);
    int* d_sT = S.get<int>((size_t)nslT + 1);
    int* d_long = S.get<int>((size_t)n);
    long long* d_sums = S.get<long long>((size_t)nb);
    long long* d_info = S.get<long long>(4);              // too long, long columns, nnz, stored entries of A'
    if (!d_rpT || !d_slT || !d_sT || !d_long || !d_sums || !d_info) return ACS_ERR_OOM;
    if (cudaMemsetAsync(d_info, 0, sizeof(long long) * 4, st) != cudaSuccess) return ACS_ERR_CUDA;
    col_slices<<<grid_for(nslT, 256), 256, 0, st>>>(n, gAT, d_cnt, d_slT, d_info, d_long);
    exclusive_scan(n, ColCount{d_cnt}, OffsetsOut{d_rpT, n}, d_sums, d_info + 2, st);
    exclusive_scan(nslT, SliceWidth{d_slT}, SlicePtrOut{d_sT, nslT}, d_sums, d_info + 3, st);
    long long info[4];
    out.slenT.resize((size_t)nslT);
    out.sptrT.resize((size_t)nslT + 1);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(info, d_info, sizeof(info), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(out.slenT.data(), d_slT, sizeof(int) * nslT, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(out.sptrT.data(), d_sT, sizeof(int) * (nslT + 1), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ACS_ERR_CUDA;
    P->d2h_bytes += (long long)sizeof(info) + 4 * (2 * nslT + 1);
    trace("tables of A'");
    if (info[0]) return 1;                                   // a column left to the host builder
    if (info[2] != nnz) return ACS_ERR_CSR;                  // cannot happen: the counts sum to nnz
    const long long nlong = info[1];
    const long long totT = info[3];
    if (totT >= INT32_MAX) return ACS_ERR_CSR;
    int* d_cur = S.get<int>(n);
    int* d_rowsT = S.get<int>((size_t)nnz);
    double* d_valsT = S.get<double>((size_t)nnz);
    int* d_sA = S.get<int>(out.sptrA.size());
    if (!d_cur || !d_rowsT || !d_valsT || !d_sA) return ACS_ERR_OOM;
    // the images themselves belong to the problem
    int *colA = nullptr, *colT = nullptr;
    double *valA = nullptr, *valT = nullptr;
    if (!P->alloc(&colA, (size_t)std::max<long long>(totA, 1)) || !P->alloc(&valA, (size_t)std::max<long long>(totA, 1)) ||
        !P->alloc(&colT, (size_t)std::max<long long>(totT, 1)) || !P->alloc(&valT, (size_t)std::max<long long>(totT, 1)))
        return ACS_ERR_OOM;
    trace("scratch and images");
    if (cudaMemcpyAsync(d_sA, out.sptrA.data(), sizeof(int) * out.sptrA.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(d_cur, 0, sizeof(int) * n, st) != cudaSuccess ||
        cudaMemsetAsync(colA, 0, sizeof(int) * totA, st) != cudaSuccess ||
        cudaMemsetAsync(valA, 0, sizeof(double) * totA, st) != cudaSuccess ||
        cudaMemsetAsync(colT, 0, sizeof(int) * totT, st) != cudaSuccess ||
        cudaMemsetAsync(valT, 0, sizeof(double) * totT, st) != cudaSuccess)
        return ACS_ERR_CUDA;
    P->h2d_bytes += 4LL * (long long)out.sptrA.size();
    trace("tables up, images zeroed");
    pack_rows<<<grid_for(32LL * m, 256), 256, 0, st>>>(m, gA, d_sA, d_begA, d_lenA, d_col, d_val, colA, valA);
    scatter_cols<<<grid_for(32LL * m, 256), 256, 0, st>>>(m, d_begA, d_lenA, d_col, d_val, d_rpT, d_cur, d_rowsT,
                                                            d_valsT);
    sort_short<<<grid_for(n, 256), 256, 0, st>>>(n, d_rpT, d_cnt, d_rowsT, d_valsT);
    if (nlong > 0) sort_long<<<(unsigned)nlong, 512, 0, st>>>(d_long, d_rpT, d_cnt, d_rowsT, d_valsT);
    pack_rows<<<grid_for(32LL * n, 256), 256, 0, st>>>(n, gAT, d_sT, d_rpT, d_cnt, d_rowsT, d_valsT, colT, valT);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return ACS_ERR_CUDA;
    trace("pack, scatter, sort");
    out.colA = colA;
    out.valA = valA;
    out.colT = colT;
    out.valT = valT;
    out.totA = totA;
    out.totT = totT;
    return ACS_SOLVED;
}

}  // namespace acs
