// KKT residuals of a caller-supplied point without any allocation.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool or under a fixed memory budget, real-time loops that
// must not enter the allocator, and drivers that hand over only pre-allocated
// buffers.  This entry point serves them: the caller passes every input and the
// output in device memory it already owns, and the temporary data of the
// computation live in one file-scope device array of fixed size that every GPU
// which loads this library holds until the process exits.
//
// Scratch layout (doubles): kMaxN entries for A'y, then kMaxBlocks x 8 block
// partials.  A'y is accumulated by scattering the rows of A (atomic adds), so
// its summation order, and hence the last bits of r_d, may differ from call to
// call.  The accumulator is cleared at the start of every call.  Calls that
// overlap on the GPU (different streams, or another thread) share the array
// and race; callers must order them.

#include <math.h>
#include <mutex>

#include "../../include/acs.h"

namespace {

constexpr int kMaxN = 1 << 20;                 // largest n accepted (1,048,576): 8 MiB of A'y
constexpr int kMaxBlocks = 1024;               // grid size of the two reduction kernels
constexpr int kVals = 8;                       // partials per block
constexpr int kThreadsNA = 256;

__device__ __align__(256) double g_noalloc_scratch[kMaxN + kMaxBlocks * kVals];

std::mutex g_setup_mutex;

__device__ __forceinline__ double warp_sum_na(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block-wide sums of NV values; thread 0 writes them to out[0..NV).
template <int NV>
__device__ void block_sum_store(double (&v)[NV], double* out) {
    __shared__ double sh[kThreadsNA / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const double x = warp_sum_na(v[k]);
        if (lane == 0) sh[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double x = 0.0;
        for (int w = 0; w < kThreadsNA / 32; ++w) x += sh[w][threadIdx.x];
        out[threadIdx.x] = x;
    }
}

// Rows of A: partials ||Ax - b||^2, b'y, ||b||^2; scatter y_i A_ij into aty[j].
__global__ void __launch_bounds__(kThreadsNA) rows_kernel(int m, const int* __restrict__ rp, const int* __restrict__ ci,
                                                          const double* __restrict__ av, const double* __restrict__ b,
                                                          const double* __restrict__ x, const double* __restrict__ y,
                                                          double* aty, double* partials) {
    double v[3] = {0.0, 0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int e = rp[i + 1];
        const double yi = y[i];
        double s = 0.0;
        for (int k = rp[i]; k < e; ++k) {
            const int j = ci[k];
            s = fma(av[k], x[j], s);
            atomicAdd(aty + j, av[k] * yi);
        }
        const double d = s - b[i];
        v[0] += d * d;
        v[1] += b[i] * yi;
        v[2] += b[i] * b[i];
    }
    block_sum_store<3>(v, partials + blockIdx.x * kVals);
}

__device__ __forceinline__ double soc_dist2_na(double v1, double t) {
    if (t <= v1) return 0.0;
    if (t <= -v1) return v1 * v1 + t * t;
    const double d = 0.5 * (t - v1);
    return 2.0 * d * d;
}

// Coordinates and cones: ||A'y + z - c||^2, c'x, ||x||^2, ||z||^2, dist(x,K)^2,
// dist(z,K)^2, ||c||^2.
__global__ void __launch_bounds__(kThreadsNA) cols_kernel(int n, int n_orth, int n_soc, const int* __restrict__ soc_off,
                                                          const double* __restrict__ c, const double* __restrict__ x,
                                                          const double* __restrict__ z, const double* aty,
                                                          double* partials) {
    double v[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double d = aty[j] + z[j] - c[j];
        v[0] += d * d;
        v[6] += c[j] * c[j];
        v[1] += c[j] * x[j];
        v[2] += x[j] * x[j];
        v[3] += z[j] * z[j];
        if (j < n_orth) {
            if (x[j] < 0.0) v[4] += x[j] * x[j];
            if (z[j] < 0.0) v[5] += z[j] * z[j];
        }
    }
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_soc; q += gridDim.x * blockDim.x) {
        const int a = soc_off[q], e = soc_off[q + 1];
        double sx = 0.0, sz = 0.0;
        for (int j = a + 1; j < e; ++j) {
            sx = fma(x[j], x[j], sx);
            sz = fma(z[j], z[j], sz);
        }
        v[4] += soc_dist2_na(x[a], sqrt(sx));
        v[5] += soc_dist2_na(z[a], sqrt(sz));
    }
    block_sum_store<7>(v, partials + blockIdx.x * kVals);
}

// One block: combine the partials in block order, write the six residual values.
__global__ void finish_kernel(int nb_rows, int nb_cols, const double* prow, const double* pcol, double* out) {
    if (threadIdx.x != 0) return;
    double rp = 0, by = 0, bb = 0, rd = 0, cx = 0, xx = 0, zz = 0, dx = 0, dz = 0, cc = 0;
    for (int k = 0; k < nb_rows; ++k) {
        rp += prow[k * kVals]; by += prow[k * kVals + 1]; bb += prow[k * kVals + 2];
    }
    for (int k = 0; k < nb_cols; ++k) {
        const double* p = pcol + k * kVals;
        rd += p[0]; cx += p[1]; xx += p[2]; zz += p[3]; dx += p[4]; dz += p[5]; cc += p[6];
    }
    const double bnorm = sqrt(bb), cnorm = sqrt(cc);
    out[0] = sqrt(rp) / (1.0 + bnorm);
    out[1] = sqrt(rd) / (1.0 + cnorm);
    out[2] = fabs(cx - by) / (1.0 + fabs(cx) + fabs(by));
    out[3] = fmax(sqrt(dx), sqrt(dz)) / (1.0 + fmax(sqrt(xx), sqrt(zz)));
    out[4] = cx;
    out[5] = by;
}

// Device address of the scratch array in the current device's context,
// looked up on every call: a lookup is a host-side table query that
// allocates nothing, and a cached address would outlive the context it
// belongs to (after cudaDeviceReset the module is loaded again elsewhere).
// The first lookup in a context loads the module; the lock keeps concurrent
// first calls from racing in the runtime's lazy loading.
double* scratch_for_current_device(int* err) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    double* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_noalloc_scratch) != cudaSuccess || !p) {
        *err = ACS_ERR_CUDA;
        return nullptr;
    }
    return p;
}

}  // namespace

extern "C" int acs_kkt_residuals_noalloc(int32_t m, int32_t n, const int32_t* row_ptr, const int32_t* col,
                                         const double* val, const double* b, const double* c, const double* x,
                                         const double* y, const double* z, int32_t n_orthant, int32_t n_soc,
                                         const int32_t* soc_offsets, double* residuals, void* cuda_stream) {
    if (m <= 0 || n <= 0 || !row_ptr || !col || !val || !b || !c || !x || !y || !z || !residuals ||
        n_orthant < 0 || n_soc < 0 || (n_soc > 0 && !soc_offsets) || n_orthant > n)
        return ACS_ERR_ARG;
    if (n > kMaxN) return ACS_ERR_LIMIT;
    // an error left by an earlier, unrelated launch is not this call's
    cudaGetLastError();
    int err = ACS_SOLVED;
    double* scratch = scratch_for_current_device(&err);
    if (!scratch) return err;
    double* aty = scratch;
    double* prow = scratch + kMaxN;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // block counts in 64-bit arithmetic (m + kThreadsNA - 1 may exceed INT32_MAX)
    const long long rows_need = ((long long)m + kThreadsNA - 1) / kThreadsNA;
    const long long cols_need = ((long long)n + kThreadsNA - 1) / kThreadsNA;
    const int nb_rows = (int)(rows_need < kMaxBlocks / 2 ? rows_need : kMaxBlocks / 2);
    const int nb_cols = (int)(cols_need < kMaxBlocks / 2 ? cols_need : kMaxBlocks / 2);
    double* pcol = prow + (kMaxBlocks / 2) * kVals;
    if (cudaMemsetAsync(aty, 0, sizeof(double) * (size_t)n, st) != cudaSuccess) return ACS_ERR_CUDA;
    rows_kernel<<<nb_rows, kThreadsNA, 0, st>>>(m, row_ptr, col, val, b, x, y, aty, prow);
    cols_kernel<<<nb_cols, kThreadsNA, 0, st>>>(n, n_orthant, n_soc, soc_offsets, c, x, z, aty, pcol);
    finish_kernel<<<1, 32, 0, st>>>(nb_rows, nb_cols, prow, pcol, residuals);
    if (cudaGetLastError() != cudaSuccess) return ACS_ERR_CUDA;
    return ACS_SOLVED;
}
