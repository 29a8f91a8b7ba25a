// Random-gather rate of the device: the quantity that bounds a sparse pass
// whose gathered vector stays in L2, against the same gathers served from
// shared memory (the column-blocked layout's source).  A benchmark of the
// library (acs_bench_gather in include/acs.h), not part of a solve.

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/acs.h"

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeInFlight = 8;          // independent gathers per thread per step
constexpr int kProbeMaxSmem = 49152;       // FP32 entries staged for the shared-memory mode

// mode 0: default global loads, 1: L2-only loads (ld.global.cg), 2: read-only
// path (ld.global.nc), 3: from a copy in shared memory.  n is a power of two
// (n <= kProbeMaxSmem for mode 3); every thread walks its own linear
// congruential sequence of indices.
__global__ void __launch_bounds__(kProbeThreads, 1)
gather_probe_kernel(const float* __restrict__ v, int n, int steps, int mode, float* out) {
    extern __shared__ __align__(16) float xs[];
    if (mode == 3) {
        for (int k = threadIdx.x; k < n; k += blockDim.x) xs[k] = v[k];
        __syncthreads();
    }
    const unsigned mask = (unsigned)n - 1u;
    unsigned x[kProbeInFlight];
#pragma unroll
    for (int u = 0; u < kProbeInFlight; ++u) x[u] = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + u * 40503u + 1u;
    float acc = 0.f;
    for (int i = 0; i < steps; ++i) {
        float g[kProbeInFlight];
#pragma unroll
        for (int u = 0; u < kProbeInFlight; ++u) {
            x[u] = x[u] * 1664525u + 1013904223u;
            const unsigned idx = (x[u] >> 8) & mask;
            if (mode == 3) g[u] = xs[idx];
            else if (mode == 1) g[u] = __ldcg(v + idx);
            else if (mode == 2) g[u] = __ldg(v + idx);
            else g[u] = v[idx];
        }
#pragma unroll
        for (int u = 0; u < kProbeInFlight; ++u) acc += g[u];
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;      // keeps the gathers
}

}  // namespace

extern "C" int acs_bench_gather(int32_t device, int64_t entries, int32_t mode, int32_t steps,
                                double* gathers_per_s) {
    if (!gathers_per_s || entries < 32 || (entries & (entries - 1)) != 0 || entries > (1LL << 24) || mode < 0 ||
        mode > 3 || steps <= 0 || (mode == 3 && entries > kProbeMaxSmem))
        return ACS_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return ACS_ERR_CUDA;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return ACS_ERR_CUDA;
    const int smem = mode == 3 ? (int)entries * (int)sizeof(float) : 0;
    if (cudaFuncSetAttribute(gather_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kProbeMaxSmem * (int)sizeof(float)) != cudaSuccess)
        return ACS_ERR_CUDA;
    float* v = nullptr;
    float* out = nullptr;
    const size_t nthreads = (size_t)nsm * kProbeThreads;
    if (cudaMalloc(&v, sizeof(float) * (size_t)entries) != cudaSuccess) return ACS_ERR_OOM;
    if (cudaMalloc(&out, sizeof(float) * nthreads) != cudaSuccess) {
        cudaFree(v);
        return ACS_ERR_OOM;
    }
    int rc = ACS_SOLVED;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    if (cudaMemset(v, 0, sizeof(float) * (size_t)entries) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = ACS_ERR_CUDA;
    } else {
        // one launch to warm L2, then the timed one
        gather_probe_kernel<<<nsm, kProbeThreads, smem>>>(v, (int)entries, steps, mode, out);
        cudaEventRecord(e0);
        gather_probe_kernel<<<nsm, kProbeThreads, smem>>>(v, (int)entries, steps, mode, out);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess)
            rc = ACS_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(v);
    cudaFree(out);
    if (rc == ACS_SOLVED) *gathers_per_s = (double)nthreads * steps * kProbeInFlight / (ms * 1e-3);
    return rc;
}
