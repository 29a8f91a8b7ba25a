// Sliced-ELLPACK images of A and A' built on the device from the caller's
// CSR (single-problem create): the same images the host builder makes
// (acs_host.cuh: build_sell, transpose_relabelled), bit for bit, with the
// host doing only O(m + n) work (slice tables, prefix sums).
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

#include <algorithm>
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
    // A: relabelled rows
    std::vector<long long> begA(m);
    std::vector<int> lenA(m);
    for (int r = 0; r < m; ++r) {
        begA[r] = row_ptr[perm[r]];
        lenA[r] = (int)(row_ptr[perm[r] + 1] - row_ptr[perm[r]]);
    }
    const long long totA = host::sell_shape(m, gA, [&](int r) { return (long long)lenA[r]; }, out.sptrA, out.slenA);
    if (totA >= INT32_MAX) return ACS_ERR_CSR;
    int* d_col = S.get<int>((size_t)nnz);
    double* d_val = S.get<double>((size_t)nnz);
    long long* d_begA = S.get<long long>(m);
    int* d_lenA = S.get<int>(m);
    int* d_cnt = S.get<int>(n);
    if (!d_col || !d_val || !d_begA || !d_lenA || !d_cnt) return ACS_ERR_OOM;
    if (cudaMemcpyAsync(d_col, col, sizeof(int) * nnz, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_val, val, sizeof(double) * nnz, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_begA, begA.data(), sizeof(long long) * m, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_lenA, lenA.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(d_cnt, 0, sizeof(int) * n, st) != cudaSuccess)
        return ACS_ERR_CUDA;
    count_cols<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, d_col, d_cnt);
    std::vector<int> cnt(n);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ACS_ERR_CUDA;
    // A': column offsets, the longer columns, the slice table
    std::vector<long long> rpT((size_t)n + 1, 0);
    std::vector<int> longc;
    for (int j = 0; j < n; ++j) {
        rpT[j + 1] = rpT[j] + cnt[j];
        if (cnt[j] > kDevSortMax) return 1;                  // left to the host builder
        if (cnt[j] > kShortSort) longc.push_back(j);
    }
    const long long totT = host::sell_shape(n, gAT, [&](int j) { return (long long)cnt[j]; }, out.sptrT, out.slenT);
    if (totT >= INT32_MAX) return ACS_ERR_CSR;
    long long* d_rpT = S.get<long long>((size_t)n + 1);
    int* d_cur = S.get<int>(n);
    int* d_rowsT = S.get<int>((size_t)nnz);
    double* d_valsT = S.get<double>((size_t)nnz);
    int* d_long = S.get<int>(longc.size());
    int* d_sA = S.get<int>(out.sptrA.size());
    int* d_sT = S.get<int>(out.sptrT.size());
    if (!d_rpT || !d_cur || !d_rowsT || !d_valsT || !d_long || !d_sA || !d_sT) return ACS_ERR_OOM;
    // the images themselves belong to the problem
    int *colA = nullptr, *colT = nullptr;
    double *valA = nullptr, *valT = nullptr;
    if (!P->alloc(&colA, (size_t)std::max<long long>(totA, 1)) || !P->alloc(&valA, (size_t)std::max<long long>(totA, 1)) ||
        !P->alloc(&colT, (size_t)std::max<long long>(totT, 1)) || !P->alloc(&valT, (size_t)std::max<long long>(totT, 1)))
        return ACS_ERR_OOM;
    if (cudaMemcpyAsync(d_rpT, rpT.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_long, longc.data(), sizeof(int) * longc.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_sA, out.sptrA.data(), sizeof(int) * out.sptrA.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_sT, out.sptrT.data(), sizeof(int) * out.sptrT.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(d_cur, 0, sizeof(int) * n, st) != cudaSuccess ||
        cudaMemsetAsync(colA, 0, sizeof(int) * totA, st) != cudaSuccess ||
        cudaMemsetAsync(valA, 0, sizeof(double) * totA, st) != cudaSuccess ||
        cudaMemsetAsync(colT, 0, sizeof(int) * totT, st) != cudaSuccess ||
        cudaMemsetAsync(valT, 0, sizeof(double) * totT, st) != cudaSuccess)
        return ACS_ERR_CUDA;
    pack_rows<<<grid_for(32LL * m, 256), 256, 0, st>>>(m, gA, d_sA, d_begA, d_lenA, d_col, d_val, colA, valA);
    scatter_cols<<<grid_for(32LL * m, 256), 256, 0, st>>>(m, d_begA, d_lenA, d_col, d_val, d_rpT, d_cur, d_rowsT,
                                                            d_valsT);
    sort_short<<<grid_for(n, 256), 256, 0, st>>>(n, d_rpT, d_cnt, d_rowsT, d_valsT);
    if (!longc.empty()) sort_long<<<(unsigned)longc.size(), 512, 0, st>>>(d_long, d_rpT, d_cnt, d_rowsT, d_valsT);
    pack_rows<<<grid_for(32LL * n, 256), 256, 0, st>>>(n, gAT, d_sT, d_rpT, d_cnt, d_rowsT, d_valsT, colT, valT);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return ACS_ERR_CUDA;
    out.colA = colA;
    out.valA = valA;
    out.colT = colT;
    out.valT = valT;
    out.totA = totA;
    out.totT = totT;
    return ACS_SOLVED;
}

}  // namespace acs
