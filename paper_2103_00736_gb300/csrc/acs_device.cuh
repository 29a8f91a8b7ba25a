// Device code of the conic solver shared by the single-problem launch
// (acs_iter.cu: one team = the whole grid) and the batched launch
// (acs_batch.cu: one team of CTAs per problem): grid/team barriers and
// reductions, sliced-ELLPACK products, the phases of Algorithm 2 and the
// solve loop.  See acs_iter.cu for the method and the precision scheme.
#pragma once

#include <math.h>
#include <stdio.h>

#include "acs_internal.cuh"

namespace acs {

// ---------------------------------------------------------------------------
// synchronisation and reductions
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(volatile const int*)p; }

// Grid-wide reduction and barrier.
//
// A phase leaves its contributions to a reduction in shared memory
// (block_partials: warp shuffles, then one warp combines the warps in fixed
// order).  grid_sync then publishes this CTA's partials followed by an
// arrival flag holding the barrier generation; thread b of every CTA waits
// for the flag of CTA b and loads CTA b's partials, and the CTA combines them
// in CTA order (a fixed shuffle tree, then the warps in order).  Every CTA
// thus computes bit-identical reduced values (deterministic for a given
// launch shape) after a single one-way flag latency.  All waits are bounded
// (kBarrierTimeoutNs): on expiry, or when another CTA has recorded an error,
// the wait records ACS_ERR_DEVICE_TIMEOUT and grid_sync returns false in
// every thread; the caller then leaves the kernel.
constexpr int kMaxGrid = 256;   // CTAs of a persistent launch (one per SM)

struct SyncShared {
    int team_rank;            // this CTA's rank in the team working on one problem
    int team_size;            // CTAs in the team (the whole grid for a single solve)
    unsigned long long* bar;  // the team's monotonic barrier arrival counter
    double* tpart;            // the team's partials, [team_size * kMaxRed]
    double* dM;               // the team's dense scratch for the cached projection operator:
    double* dX;               //   M / its Cholesky factor and L^{-1}, [m * m] each
    unsigned long long deadline;  // global-timer time at which a time-sliced solve pauses (0 = none)
    double blk[kMaxRed];      // this CTA's partials
    double out[kMaxRed];      // grid-reduced values of the last barrier
    double wsum[kWarps][kMaxRed];
    double gath[kMaxRed][kMaxGrid];   // every CTA's partials, gathered
    int op[kMaxRed];          // 0 = sum, 1 = max
    int nv;                   // number of values reduced at the next barrier
    int fail;
    unsigned gen;             // barrier generation (same sequence in every CTA)
    // column-blocked passes: the mbarrier that completes a block's bulk copy
    // into shared memory, and its phase parity (flips once per block staged)
    unsigned long long stage_bar;
    unsigned stage_phase;
    int cb_next;              // next run of the current segment to deal to a warp
    // the combine phases' two tile slots: their mbarriers and phase parities
    unsigned long long comb_bar[2];
    unsigned comb_phase[2];
};

__device__ __forceinline__ SyncShared& sync_smem() {
    __shared__ SyncShared s;
    return s;
}

// A team is the set of CTAs that work on one problem: the whole grid of a
// single-problem launch, or a group of CTAs (often one) of a batched launch.
// Phases index coordinates, rows and cones by the thread's rank in its team.
__device__ __forceinline__ void team_set(int rank, int size, unsigned long long* bar, double* partials,
                                         double* dense_M = nullptr, double* dense_X = nullptr) {
    SyncShared& S = sync_smem();
    if (threadIdx.x == 0) {
        S.team_rank = rank;
        S.team_size = size;
        S.bar = bar;
        S.tpart = partials;
        S.dM = dense_M;
        S.dX = dense_X;
        S.deadline = 0ull;
    }
    __syncthreads();
}
__device__ __forceinline__ int team_rank() { return sync_smem().team_rank; }
__device__ __forceinline__ int team_size() { return sync_smem().team_size; }
__device__ __forceinline__ int global_tid() { return team_rank() * (int)blockDim.x + (int)threadIdx.x; }
__device__ __forceinline__ int global_threads() { return team_size() * (int)blockDim.x; }
__device__ __forceinline__ int global_warp() { return global_tid() >> 5; }
__device__ __forceinline__ int global_warps() { return global_threads() >> 5; }

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Stage this CTA's contribution to the values reduced at the next grid_sync.
template <int NV>
__device__ void block_partials(const double (&v)[NV], const int (&op)[NV], double* /*unused*/) {
    SyncShared& S = sync_smem();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const double x = op[k] ? warp_max(v[k]) : warp_sum(v[k]);
        if (lane == 0) S.wsum[warp][k] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = (lane < (int)(blockDim.x >> 5)) ? S.wsum[lane][k] : (op[k] ? -INFINITY : 0.0);
            x = op[k] ? warp_max(x) : warp_sum(x);
            if (lane == 0) {
                S.blk[k] = x;
                S.op[k] = op[k];
            }
        }
        if (lane == 0) S.nv = NV;
    }
}

// Start (or resume, with the generation reached so far) the team's barrier
// sequence and clear the failure flag.
static __device__ void sync_init(unsigned gen) {
    SyncShared& S = sync_smem();
    if (threadIdx.x == 0) {
        S.nv = 0;
        S.fail = 0;
        S.gen = gen;
    }
    __syncthreads();
}

__device__ __forceinline__ void red_add_release(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Barrier: thread 0 of every CTA of the team publishes the CTA's partials,
// adds 1 to the team's monotonic arrival counter with release semantics and
// spins (acquire) until the counter reaches (generation) * (CTAs in the team).
// A team of one CTA needs no counter: its partials are already combined.  One thread per CTA polls a
// single word, which keeps the barrier at about the latency of two L2 round
// trips.  The partials of all CTAs are then read once, in parallel.
static __device__ __noinline__ bool grid_sync(int* err) {
    SyncShared& S = sync_smem();
    __syncthreads();                                   // the phase's writes and S.blk are complete
    const unsigned target = S.gen + 1u;
    const int nv = S.nv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rank = S.team_rank, size = S.team_size;
    if (size == 1) {
        // writes of the phase are visible to the CTA after __syncthreads; the
        // error word is still checked so that a failed problem stops
        if (threadIdx.x == 0) {
            for (int k = 0; k < nv; ++k) S.out[k] = S.blk[k];
            if (ld_volatile_int(err) != 0) S.fail = 1;
        }
        __syncthreads();
        const bool ok1 = S.fail == 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            S.gen = target;
            S.nv = 0;
        }
        return ok1;
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < nv; ++k) S.tpart[rank * kMaxRed + k] = S.blk[k];
        red_add_release(S.bar, 1ull);
        const unsigned long long want = (unsigned long long)target * size;
        const unsigned long long t0 = gtimer();
        int spins = 0;
        while (ld_acquire64(S.bar) < want) {
            if (++spins == 64) {
                spins = 0;
                if (ld_volatile_int(err) != 0) { S.fail = 1; break; }
                if (gtimer() - t0 > kBarrierTimeoutNs) {
                    atomicCAS(err, 0, ACS_ERR_DEVICE_TIMEOUT);
                    S.fail = 1;
                    break;
                }
            }
        }
        if (ld_volatile_int(err) != 0) S.fail = 1;
    }
    __syncthreads();
    if (nv > 0) {
        // gather every CTA's partials, combine in CTA order: lanes by a fixed
        // shuffle tree, then the warps in order
        const int b = threadIdx.x;
        if (b < size)
            for (int k = 0; k < nv; ++k) S.gath[k][b] = __ldcg(S.tpart + b * kMaxRed + k);
        __syncthreads();
        const int nwarp = (size + 31) >> 5;
        if (warp < nwarp) {
            for (int k = 0; k < nv; ++k) {
                const int opk = S.op[k];
                double x = (b < size) ? S.gath[k][b] : (opk ? -INFINITY : 0.0);
                x = opk ? warp_max(x) : warp_sum(x);
                if (lane == 0) S.wsum[warp][k] = x;
            }
        }
        __syncthreads();
        if (threadIdx.x < nv) {
            const int k = threadIdx.x;
            const int opk = S.op[k];
            double x = S.wsum[0][k];
            for (int w = 1; w < nwarp; ++w) x = opk ? fmax(x, S.wsum[w][k]) : x + S.wsum[w][k];
            S.out[k] = x;
        }
    }
    __syncthreads();
    const bool ok = S.fail == 0;
    __syncthreads();                                   // everyone has read S.fail and S.out is final
    if (threadIdx.x == 0) {
        S.gen = target;
        S.nv = 0;
    }
    return ok;
}

// Values reduced at the last grid_sync.
template <int NV>
__device__ void grid_combine(const double* /*unused*/, const int (&)[NV], double (&out)[NV]) {
    SyncShared& S = sync_smem();
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = S.out[k];
}

// ---------------------------------------------------------------------------
// row-parallel sparse products (sliced ELLPACK with G lanes per row)
// ---------------------------------------------------------------------------

// Matrix entries are read once per pass: stream them past L1.
__device__ __forceinline__ int ld_stream(const int* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }

template <typename T> __device__ __forceinline__ const T* sell_vals(const SellMat& M);
template <> __device__ __forceinline__ const float* sell_vals<float>(const SellMat& M) { return M.v32; }
template <> __device__ __forceinline__ const double* sell_vals<double>(const SellMat& M) { return M.v64; }

// Stored value -> arithmetic type.  A BF16 value is the upper half of the
// FP32 value with the same bits, so the conversion is exact.
__device__ __forceinline__ unsigned short ld_stream(const unsigned short* p) { return __ldcs(p); }
template <typename T> __device__ __forceinline__ T val_to(T v) { return v; }
template <typename T> __device__ __forceinline__ T val_to(unsigned short b);
template <> __device__ __forceinline__ float val_to<float>(unsigned short b) {
    return __uint_as_float((unsigned)b << 16);
}

// Layout (see SellMat): a slice holds 32/G rows; chunk c of the slice is 32
// consecutive entries, entry k of local row r at chunk k/G, lane r*G + k%G.
// Warp w handles slices w, w + nwarps, ..., in batches of U chunks; each lane
// accumulates its entries in chunk order, and the G partial sums of a row are
// combined by a fixed shuffle tree, so the result does not depend on the
// launch shape.  epi(row, sum) runs once per real row.
//
// Software pipeline: the column/value loads of the next batch (and the slice
// table entries of the next slice) are issued before the gathers of the
// current batch, so a warp keeps one matrix round trip and one gather round
// trip in flight at the same time instead of one after the other.
template <int U, typename T, typename V>
__device__ __forceinline__ void sell_load_batch(const int* __restrict__ col, const V* __restrict__ val,
                                                int base, int k, int len, int (&c)[U], T (&a)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (k + u < len) {
            c[u] = ld_stream(col + base + 32 * (k + u));
            a[u] = val_to<T>(ld_stream(val + base + 32 * (k + u)));
        } else {
            c[u] = 0;
            a[u] = T(0);
        }
    }
}

// V: the stored value type (T itself, or BF16 bits for T = float).
template <int G, int U, typename T, typename V, typename Gather, typename Epi>
__device__ __forceinline__ void sell_rows_g(const SellMat& M, const V* __restrict__ val, Gather gather, Epi epi) {
    const int* __restrict__ col = M.col;
    const int lane = threadIdx.x & 31;
    const int nw = global_warps();
    int sl = global_warp();
    if (sl >= M.nslices) return;                        // warp-uniform
    int len = __ldg(M.slen + sl);
    int base = __ldg(M.sptr + sl) + lane;
    int k = 0;
    // slice table entries of the following slice, loaded one slice ahead
    int nsl = sl + nw;
    int nlen = 0, nbase = 0;
    if (nsl < M.nslices) {
        nlen = __ldg(M.slen + nsl);
        nbase = __ldg(M.sptr + nsl) + lane;
    }
    int c[U];
    T a[U];
    sell_load_batch<U>(col, val, base, k, len, c, a);
    T acc = T(0);
    while (true) {
        // next batch: more chunks of this slice, or the first of the next slice
        const bool same = k + U < len;
        const bool have_next = same || nsl < M.nslices;
        int c2[U];
        T a2[U];
        if (same) sell_load_batch<U>(col, val, base, k + U, len, c2, a2);
        else if (have_next) sell_load_batch<U>(col, val, nbase, 0, nlen, c2, a2);
        T x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = gather(c[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) acc = fma(a[u], x[u], acc);
        if (!same) {                                    // slice finished
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            const int row = sl * (32 / G) + lane / G;
            if ((lane & (G - 1)) == 0 && row < M.nrows) epi(row, acc);
            acc = T(0);
            if (!have_next) break;
            sl = nsl;
            len = nlen;
            base = nbase;
            k = 0;
            nsl = sl + nw;
            if (nsl < M.nslices) {
                nlen = __ldg(M.slen + nsl);
                nbase = __ldg(M.sptr + nsl) + lane;
            }
        } else {
            k += U;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            c[u] = c2[u];
            a[u] = a2[u];
        }
    }
}

// Chunks per software-pipeline batch: each lane keeps U column/value loads
// and U gathers in flight.  Measured on the large LP (1e7 nonzeros): U = 4,
// 8, 12 give 58.9, 57.9, 70.1 us for the CG A pass and 44.8, 46.2, 51.2 us
// for the A' pass -- the passes are bound by the L2 gather rate, not by the
// depth of the chain -- so 4 stays; FP64 passes at 8 would spill registers.
#ifndef ACS_CG_U
#define ACS_CG_U 4
#endif

template <typename T, typename V, typename Gather, typename Epi>
__device__ __forceinline__ void sell_rows_v(const SellMat& M, const V* val, Gather gather, Epi epi) {
    constexpr int U = (sizeof(T) == 4) ? ACS_CG_U : 4;
    switch (M.g) {
        case 1: sell_rows_g<1, U, T>(M, val, gather, epi); break;
        case 2: sell_rows_g<2, U, T>(M, val, gather, epi); break;
        case 4: sell_rows_g<4, U, T>(M, val, gather, epi); break;
        case 8: sell_rows_g<8, U, T>(M, val, gather, epi); break;
        case 16: sell_rows_g<16, U, T>(M, val, gather, epi); break;
        default: sell_rows_g<32, U, T>(M, val, gather, epi); break;
    }
}

// FP32 products read the BF16 copy of the values when A is stored in BF16.
template <typename T, typename Gather, typename Epi>
__device__ __forceinline__ void sell_rows(const SellMat& M, Gather gather, Epi epi) {
    if (sizeof(T) == 4 && M.v16 != nullptr) sell_rows_v<T>(M, M.v16, gather, epi);
    else sell_rows_v<T>(M, sell_vals<T>(M), gather, epi);
}

// Two sums per row: sum a*g1(j) and sum a*a*g2(j) (FP64 values).
template <int G, typename G1, typename G2, typename Epi>
__device__ __forceinline__ void sell_rows2_g(const SellMat& M, G1 g1, G2 g2, Epi epi) {
    const int lane = threadIdx.x & 31;
    const int nw = global_warps();
    for (int sl = global_warp(); sl < M.nslices; sl += nw) {
        const int len = __ldg(M.slen + sl);
        int idx = __ldg(M.sptr + sl) + lane;
        double acc1 = 0.0, acc2 = 0.0;
        for (int k = 0; k < len; ++k, idx += 32) {
            const int j = ld_stream(M.col + idx);
            const double a = ld_stream(M.v64 + idx);
            acc1 = fma(a, g1(j), acc1);
            acc2 = fma(a * a, g2(j), acc2);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
            acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
        }
        const int row = sl * (32 / G) + lane / G;
        if ((lane & (G - 1)) == 0 && row < M.nrows) epi(row, acc1, acc2);
    }
}

template <typename G1, typename G2, typename Epi>
__device__ __forceinline__ void sell_rows2(const SellMat& M, G1 g1, G2 g2, Epi epi) {
    switch (M.g) {
        case 1: sell_rows2_g<1>(M, g1, g2, epi); break;
        case 2: sell_rows2_g<2>(M, g1, g2, epi); break;
        case 4: sell_rows2_g<4>(M, g1, g2, epi); break;
        case 8: sell_rows2_g<8>(M, g1, g2, epi); break;
        case 16: sell_rows2_g<16>(M, g1, g2, epi); break;
        default: sell_rows2_g<32>(M, g1, g2, epi); break;
    }
}

// ---------------------------------------------------------------------------
// column-blocked products (layout in acs_internal.cuh / acs_cbsell.cuh)
// ---------------------------------------------------------------------------

// Dynamic shared memory of the single-problem FP32 launch: the block of the
// multiplied vector that a column-blocked pass gathers from.
extern __shared__ __align__(16) float acs_cb_smem[];

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// Set up the staging barrier (once per launch, before the first pass).
__device__ __forceinline__ void cb_init() {
    SyncShared& S = sync_smem();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.stage_bar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.comb_bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.comb_bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.stage_phase = 0u;
        S.comb_phase[0] = S.comb_phase[1] = 0u;
    }
    __syncthreads();
}

// Bounded wait for the staging barrier's current phase (2 s, then the error
// word records ACS_ERR_DEVICE_TIMEOUT; the next grid barrier ends the launch).
__device__ __forceinline__ bool cb_wait_bar(unsigned long long* mbar, unsigned parity, int* err) {
    const unsigned bar = smem_u32(mbar);
    unsigned done = 0;
    const unsigned long long t0 = gtimer();
    int spins = 0;
    while (true) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (++spins == 64) {
            spins = 0;
            if (gtimer() - t0 > kBarrierTimeoutNs) {
                atomicCAS(err, 0, ACS_ERR_DEVICE_TIMEOUT);
                return false;
            }
        }
    }
}

// Stage x[c0, c0 + w) in shared memory as FP32.  The vector was written by
// other CTAs before the last grid barrier.  An FP32 vector is copied by the
// bulk-copy engine: thread 0 issues 1-D bulk copies (16-byte multiples; c0 is
// a multiple of 4 and the vector 16-byte aligned) that complete on the
// staging mbarrier, the last w mod 4 entries by plain loads; an FP64 vector
// is read and rounded by all threads, eight loads in flight per thread.
template <typename Src>
__device__ __forceinline__ void cb_stage(float* xs, const Src* __restrict__ x, int c0, int w, int* err) {
    SyncShared& S = sync_smem();
    if constexpr (sizeof(Src) == 4) {
        const int w4 = w & ~3;
        const unsigned parity = S.stage_phase;
        if (w4 > 0 && threadIdx.x == 0) {
            const unsigned bar = smem_u32(&S.stage_bar);
            const unsigned bytes = (unsigned)w4 * 4u;
            // generic-proxy writes to x (other CTAs, before the grid barrier)
            // and generic reads of xs (before the CTA barrier) come first
            asm volatile("fence.proxy.async.global;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                         : "memory");
            constexpr unsigned kChunk = 32768u;
            const char* src = reinterpret_cast<const char*>(x + c0);
            char* dst = reinterpret_cast<char*>(xs);
            for (unsigned o = 0; o < bytes; o += kChunk) {
                const unsigned len = bytes - o < kChunk ? bytes - o : kChunk;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(dst + o)),
                    "l"(src + o), "r"(len), "r"(bar)
                    : "memory");
            }
        }
        for (int k = w4 + (int)threadIdx.x; k < w; k += blockDim.x) xs[k] = __ldcg(x + c0 + k);
        if (w4 > 0) {
            cb_wait_bar(&S.stage_bar, parity, err);
            __syncthreads();                             // every thread has seen the phase
            if (threadIdx.x == 0) S.stage_phase = parity ^ 1u;
        }
    } else {
        constexpr int kIn = 8;
        const int step = (int)blockDim.x * kIn;
        for (int k0 = threadIdx.x; k0 < w; k0 += step) {
            double v[kIn];
#pragma unroll
            for (int u = 0; u < kIn; ++u) {
                const int k = k0 + u * (int)blockDim.x;
                v[u] = k < w ? __ldcg(x + c0 + k) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kIn; ++u) {
                const int k = k0 + u * (int)blockDim.x;
                if (k < w) xs[k] = (float)v[u];
            }
        }
    }
}

template <int U>
__device__ __forceinline__ void cb_load_batch(const unsigned short* __restrict__ col, const float* __restrict__ val,
                                              int base, int k, int len, unsigned (&c)[U], float (&a)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (k + u < len) {
            c[u] = __ldcs(col + base + 32 * (k + u));
            a[u] = __ldcs(val + base + 32 * (k + u));
        } else {
            c[u] = 0u;
            a[u] = 0.f;
        }
    }
}

// Items are multiplied in runs of kCbRun consecutive items, whose entries
// are contiguous: a warp streams a run as one sequence of chunks (lane r of
// chunk c at 32 c + r), whatever the items' lengths, so the next batch of
// column/value loads can always be issued before the current gathers --
// across item and run boundaries.  An item ends at the chunk its end mark
// flags (every item has one).  Runs are dealt to the warps as they ask for
// them (a shared counter): the items of a window are sorted by length, so a
// fixed deal would give some warps the long runs every time.  Which warp
// multiplies a run does not change its sums.
constexpr int kCbRun = 4;

// The next run for this warp (lane 0 takes it from the counter).
__device__ __forceinline__ int cb_take_run(int lane) {
    int r = 0;
    if (lane == 0) r = atomicAdd(&sync_smem().cb_next, 1);
    return __shfl_sync(0xffffffffu, r, 0);
}

// Chunks [c0, c1) of run `run` of the segment [s0, s1) (lanes 0 and 1 load
// the two offsets).
__device__ __forceinline__ void cb_run_chunks(const int* __restrict__ sptr, int s0, int s1, int run, int lane,
                                              int& c0, int& c1) {
    const int i0 = s0 + run * kCbRun;
    const int i1 = min(s1, i0 + kCbRun);
    const int v = lane < 2 ? __ldg(sptr + (lane == 0 ? i0 : i1)) : 0;
    c0 = __shfl_sync(0xffffffffu, v, 0) >> 5;
    c1 = __shfl_sync(0xffffffffu, v, 1) >> 5;
}

// End marks of chunks [c, c + U) as the low U bits (U <= 32).
template <int U>
__device__ __forceinline__ unsigned cb_marks(const unsigned* __restrict__ cend, int c) {
    const unsigned w0 = __ldg(cend + (c >> 5)), w1 = __ldg(cend + (c >> 5) + 1);
    const unsigned long long w = ((unsigned long long)w1 << 32) | w0;
    return (unsigned)(w >> (c & 31)) & ((1u << U) - 1u);
}

// U chunks starting at chunk c: lane r's entries of chunks c .. c + U - 1,
// those at or past chunk c1 read as (column 0, value 0).
template <int U>
__device__ __forceinline__ void cb_load_chunks(const unsigned short* __restrict__ col,
                                               const float* __restrict__ val, int c, int c1,
                                               unsigned (&cc)[U], float (&a)[U]) {
    const size_t e = (size_t)c * 32 + (threadIdx.x & 31);
    const unsigned short* cp = col + e;
    const float* vp = val + e;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const bool in = c + u < c1;
        cc[u] = in ? __ldcs(cp + 32 * u) : 0u;
        a[u] = in ? __ldcs(vp + 32 * u) : 0.f;
    }
}

// The items [s0, s1) of one block (one CTA's segment), in runs dealt to the
// warps as above: lane r accumulates its row's entries of each item in chunk
// order (FP32, gathers from the staged block xs) and writes the sum to
// part[item * 32 + r] (slot order: one coalesced store per item; the combine
// phases put the rows back in order).  MODE (benchmark variants): 0 the
// pass, 1 the matrix stream without the gathers, 2 without staging first.
template <int U, int MODE = 0>
__device__ __forceinline__ void cb_items(const CbMat& M, const float* xs, int s0, int s1, int warp) {
    const int nruns = (s1 - s0 + kCbRun - 1) / kCbRun;
    int run = warp;                                      // the first runs: one per warp
    if (run >= nruns) return;                            // warp-uniform
    const int lane = threadIdx.x & 31;
    int item = s0 + run * kCbRun;                        // item the next chunk belongs to
    int c, c1;                                           // chunks of the current run
    cb_run_chunks(M.sptr, s0, s1, run, lane, c, c1);
    int nrun = cb_take_run(lane), nc = 0, nc1 = 0;       // the following run, one run ahead
    if (nrun < nruns) cb_run_chunks(M.sptr, s0, s1, nrun, lane, nc, nc1);
    unsigned cc[U];
    float a[U];
    cb_load_chunks<U>(M.col, M.val, c, c1, cc, a);
    unsigned marks = cb_marks<U>(M.cend, c);
    float acc = 0.f;
    while (true) {
        const bool same = c + U < c1;
        const bool have_next = same || nrun < nruns;
        const int cn = same ? c + U : nc;                // first chunk of the next batch
        const int cn1 = same ? c1 : nc1;
        unsigned cc2[U];
        float a2[U];
        cb_load_chunks<U>(M.col, M.val, cn, have_next ? cn1 : cn, cc2, a2);
        const unsigned marks2 = have_next ? cb_marks<U>(M.cend, cn) : 0u;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (c + u < c1) {                            // warp-uniform
                if (MODE == 1) acc += a[u] + (float)cc[u];
                else acc = fmaf(a[u], xs[cc[u]], acc);
                if (marks & (1u << u)) {                 // the item ends at this chunk
                    __stcg(M.part + (size_t)item * 32 + lane, acc);
                    acc = 0.f;
                    ++item;
                }
            }
        }
        if (!have_next) break;
        if (!same) {                                     // the next run
            item = s0 + nrun * kCbRun;
            nrun = cb_take_run(lane);
            if (nrun < nruns) cb_run_chunks(M.sptr, s0, s1, nrun, lane, nc, nc1);
        }
        c = cn;
        c1 = cn1;
        marks = marks2;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cc[u] = cc2[u];
            a[u] = a2[u];
        }
    }
}

// One column-blocked pass over the items dealt to this CTA: for each block
// its range touches, stage the block of x, then multiply the range's items
// of that block.  Every slot of every item gets its sum written (0 for a row
// with no entry in the block).  Run by all threads of the CTA, after cb_init
// in the launch.
#ifndef ACS_CB_U
#define ACS_CB_U 6
#endif
template <typename Src, int MODE = 0>
__device__ __forceinline__ void cb_pass(const CbMat& M, const Src* __restrict__ x, int* err) {
    float* xs = acs_cb_smem;
    const int rank = team_rank();
    const int end = __ldg(M.cta_beg + rank + 1);
    int it = __ldg(M.cta_beg + rank);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (MODE >= 3) {
        // benchmark variants: the CTA's entries as one linear stream, chunk c
        // to warp c mod nw (3: columns and values, 4: values only)
        const int c0 = __ldg(M.sptr + it) >> 5, c1 = __ldg(M.sptr + end) >> 5;
        float acc = 0.f;
        for (int c = c0 + warp; c < c1; c += 4 * nw) {
            float v[4];
            unsigned cc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int ch = c + u * nw;
                const size_t idx = (size_t)ch * 32 + lane;
                v[u] = ch < c1 ? __ldcs(M.val + idx) : 0.f;
                cc[u] = (MODE == 3 && ch < c1) ? __ldcs(M.col + idx) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) acc += v[u] + (float)cc[u];
        }
        M.part[(size_t)(rank * nw + warp) * 32 + lane] = acc;
        return;
    }
    while (it < end) {                                   // CTA-uniform
        const int b = it / M.nsl;
        const int bend = min(end, (b + 1) * M.nsl);
        const int c0 = b * M.width;
        __syncthreads();                                 // gathers from the previous block are done
        if (threadIdx.x == 0) sync_smem().cb_next = nw;  // runs after the first one per warp
        if (MODE == 0) cb_stage(xs, x, c0, min(M.ncols - c0, M.width), err);
        __syncthreads();
        cb_items<ACS_CB_U, MODE>(M, xs, it, bend, warp);
        it = bend;
    }
}

// Dynamic shared memory of the launch (bytes).
__device__ __forceinline__ unsigned dyn_smem_bytes() {
    unsigned v;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}

// Blocks of one combine tile that fit two tile slots in `smem` bytes (at
// least 1).
__host__ __device__ __forceinline__ int cb_combine_group(int nblocks, unsigned smem) {
    const unsigned per = (unsigned)kCbWindow * 6u;       // one block's sums and slot indices of a window
    int g = (int)(smem / (2u * per));
    if (g > nblocks) g = nblocks;
    return g < 1 ? 1 : g;
}

// Adds up the partial sums of the last pass row by row, in block order, and
// calls epi(row, sum) once for every row.  A CTA takes windows of kCbWindow
// rows (rank, rank + CTAs, ...); a tile is one window and a group of G
// blocks: for each block of the group, the window's partial sums (slot
// order) and the slot of each of its rows (ipos, row order) are copied into
// one of two tile slots in shared memory by the bulk-copy engine while the
// threads work on the previous tile.  Thread k owns rows k, k + blockDim, ...
// of the window and adds their sums block after block in registers, reading
// each at its slot.  Shared memory: the two slots (needs 24 KB for G = 1).
// Run by all threads of the CTA, after cb_init in the launch.
constexpr int kCbRowsPerThread = kCbWindow / kThreads;
template <typename Epi>
__device__ __forceinline__ void cb_combine(const CbMat& M, int* err, Epi epi) {
    SyncShared& S = sync_smem();
    const int R = M.nrows, nb = M.nblocks;
    const size_t slab = (size_t)M.nsl * 32;              // slots of one block
    const int nwin = (R + kCbWindow - 1) / kCbWindow;
    const int rank = team_rank(), size = team_size();
    if (rank >= nwin) return;                            // CTA-uniform
    const int G = cb_combine_group(nb, dyn_smem_bytes());
    const int ngroups = (nb + G - 1) / G;
    const int T = ((nwin - 1 - rank) / size + 1) * ngroups;
    char* slots = reinterpret_cast<char*>(acs_cb_smem);
    const unsigned slot_bytes = (unsigned)G * kCbWindow * 6u;
    // tile t: window rank + (t / ngroups) * size, blocks of group t % ngroups
    auto issue = [&](int t) {                            // thread 0
        const int w = rank + (t / ngroups) * size, g = t % ngroups;
        const int r0 = w * kCbWindow, nslots = (min(kCbWindow, R - r0) + 31) & ~31;
        const int b0 = g * G, gb = min(G, nb - b0);
        char* sl = slots + (t & 1) * slot_bytes;
        const unsigned bar = smem_u32(&S.comb_bar[t & 1]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((unsigned)(gb * nslots * 6))
                     : "memory");
        for (int k = 0; k < gb; ++k) {
            const size_t src = (size_t)(b0 + k) * slab + (size_t)r0;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(sl + (size_t)k * kCbWindow * 4)),
                "l"(M.part + src), "r"((unsigned)nslots * 4u), "r"(bar)
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(sl + (size_t)G * kCbWindow * 4 + (size_t)k * kCbWindow * 2)),
                "l"(M.ipos + src), "r"((unsigned)nslots * 2u), "r"(bar)
                : "memory");
        }
    };
    if (threadIdx.x == 0) {
        // the partial sums were written by other CTAs before the grid barrier
        asm volatile("fence.proxy.async.global;" ::: "memory");
        issue(0);
    }
    float acc[kCbRowsPerThread];
    for (int t = 0; t < T; ++t) {
        // slot (t + 1) & 1 was last read in tile t - 1, which ended with a CTA barrier
        if (threadIdx.x == 0 && t + 1 < T) issue(t + 1);
        const int w = rank + (t / ngroups) * size, g = t % ngroups;
        const int r0 = w * kCbWindow, rows = min(kCbWindow, R - r0);
        const int b0 = g * G, gb = min(G, nb - b0);
        const unsigned parity = S.comb_phase[t & 1];
        cb_wait_bar(&S.comb_bar[t & 1], parity, err);
        const float* sp = reinterpret_cast<const float*>(slots + (t & 1) * slot_bytes);
        const unsigned short* si =
            reinterpret_cast<const unsigned short*>(slots + (t & 1) * slot_bytes + (size_t)G * kCbWindow * 4);
#pragma unroll
        for (int i = 0; i < kCbRowsPerThread; ++i) {
            const int j = (int)threadIdx.x + i * kThreads;
            float a = b0 == 0 ? 0.f : acc[i];
            if (j < rows)
                for (int k = 0; k < gb; ++k) {
                    const float v = sp[k * kCbWindow + si[k * kCbWindow + j]];
                    a = (b0 + k == 0) ? v : a + v;
                }
            acc[i] = a;
        }
        __syncthreads();                                 // the slot may be refilled
        if (threadIdx.x == 0) S.comb_phase[t & 1] = parity ^ 1u;
        if (g == ngroups - 1) {                          // the window is complete
#pragma unroll
            for (int i = 0; i < kCbRowsPerThread; ++i) {
                const int j = (int)threadIdx.x + i * kThreads;
                if (j < rows) epi(r0 + j, acc[i]);
            }
        }
    }
}

// The staging of a column-blocked pass alone (every block the CTA's range
// touches, no products): the benchmark's measure of the copy cost.
template <typename Src>
__device__ __forceinline__ void cb_stage_only(const CbMat& M, const Src* __restrict__ x, int* err) {
    float* xs = acs_cb_smem;
    const int rank = team_rank();
    const int end = __ldg(M.cta_beg + rank + 1);
    int it = __ldg(M.cta_beg + rank);
    while (it < end) {
        const int b = it / M.nsl;
        const int c0 = b * M.width;
        __syncthreads();
        cb_stage(xs, x, c0, min(M.ncols - c0, M.width), err);
        __syncthreads();
        it = min(end, (b + 1) * M.nsl);
    }
}


// ---------------------------------------------------------------------------
// cone helpers
// ---------------------------------------------------------------------------


template <typename T>
__device__ __forceinline__ T warp_sum_t(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Is iteration l in the schedule L (Algorithm 2 step 4, without the {1})?
template <typename T>
__device__ __forceinline__ bool in_schedule(const IterParams<T>& P, int l) {
    for (int i = 0; i < P.n_cond_list; ++i)
        if (__ldg(P.cond_list + i) == l) return true;
    if (P.cond_first > 0 && l >= P.cond_first) {
        if (P.cond_period <= 0) return l == P.cond_first;
        return (l - P.cond_first) % P.cond_period == 0;
    }
    return false;
}

// ---------------------------------------------------------------------------
// phases
// ---------------------------------------------------------------------------

// Conditioning, steps 5-10: o per cone, o = |x_h - ||xbar||| / |z_h|, stored
// as log o (log 0 = -inf, log inf = inf, nan stays nan); partials over the
// finite positive o: max log o, max(-log o), and their count.
template <typename T>
__device__ __noinline__ void phase_cond_o(const IterParams<T>& P) {
    double vmax = -INFINITY, vneg = -INFINITY, good = 0.0;
    for (int j = global_tid(); j < P.n_orth; j += global_threads()) {
        const double o = fabs(P.x[j]) / fabs(P.z[j]);
        const double lo = log(o);
        P.ocone[j] = lo;
        if (o > 0.0 && o < INFINITY) {
            good += 1.0;
            vmax = fmax(vmax, lo);
            vneg = fmax(vneg, -lo);
        }
    }
    const int lane = threadIdx.x & 31;
    for (int cI = global_warp(); cI < P.n_soc; cI += global_warps()) {
        const int a = __ldg(P.soc_off + cI), e = __ldg(P.soc_off + cI + 1);
        double ss = 0.0;
        for (int j = a + 1 + lane; j < e; j += 32) ss = fma(P.x[j], P.x[j], ss);
        ss = warp_sum(ss);
        if (lane == 0) {
            const double o = fabs(P.x[a] - sqrt(ss)) / fabs(P.z[a]);
            const double lo = log(o);
            P.ocone[P.n_orth + cI] = lo;
            if (o > 0.0 && o < INFINITY) {
                good += 1.0;
                vmax = fmax(vmax, lo);
                vneg = fmax(vneg, -lo);
            }
        }
    }
    const double v[3] = {vmax, vneg, good};
    const int op[3] = {1, 1, 0};
    block_partials<3>(v, op, P.partials);
}

// Exponent range of step 11 over the finite positive o.  An o of 0, inf or
// nan (x_h = ||xbar||, z_h = 0, or both) carries no scale: it takes the
// limit of the rule under the e^t cap -- the smallest scale for o = 0, the
// largest for o = inf, the geometric middle for nan.  With no finite
// positive o at all, O = I.
struct CondRange {
    double alpha, lmin, lmax;
    bool any;
};
__device__ __forceinline__ double cond_scale(double lo, const CondRange& R) {
    if (!R.any) return 1.0;
    double e = lo;
    if (isnan(lo)) e = 0.5 * (R.lmin + R.lmax);
    else if (lo == -INFINITY) e = R.lmin;
    else if (lo == INFINITY) e = R.lmax;
    return exp(R.alpha * e);
}

// Steps 11-14 per coordinate: O = exp(alpha log o) (see cond_scale),
// c_hat = O c, s = x/O - mu O z; g = O c_hat (input of the b_tilde pass).
template <typename T>
__device__ __forceinline__ void cond_apply_coord(const IterParams<T>& P, int j, double Oj, bool recast) {
    P.X.O[j] = Oj;
    P.V.O2[j] = (T)(Oj * Oj);
    const double ch = Oj * P.c[j];
    P.X.chat[j] = ch;
    P.X.g[j] = Oj * ch;
    if (recast) P.X.s[j] = P.x[j] / Oj - P.mu * Oj * P.z[j];
}

template <typename T>
__device__ __noinline__ void phase_cond_apply(const IterParams<T>& P, const CondRange& R, bool recompute_O,
                                              bool recast) {
    for (int j = global_tid(); j < P.n_orth; j += global_threads()) {
        const double Oj = recompute_O ? cond_scale(P.ocone[j], R) : P.X.O[j];
        cond_apply_coord(P, j, Oj, recast);
    }
    const int lane = threadIdx.x & 31;
    for (int cI = global_warp(); cI < P.n_soc; cI += global_warps()) {
        const int a = __ldg(P.soc_off + cI), e = __ldg(P.soc_off + cI + 1);
        const double Oc = recompute_O ? cond_scale(P.ocone[P.n_orth + cI], R) : P.X.O[a];
        for (int j = a + lane; j < e; j += 32) cond_apply_coord(P, j, Oc, recast);
    }
}

// b_tilde = b + mu A (O c_hat), J^{-1} = 1 / diag(A_hat A_hat') (FP64 pass);
// partial count of nonpositive diagonal entries.
template <typename T>
__device__ __noinline__ void phase_btilde(const IterParams<T>& P) {
    double bad = 0.0;
    const double* g = P.X.g;
    const double* O = P.X.O;
    auto g1 = [g](int j) { return g[j]; };
    auto g2 = [O](int j) { const double o = O[j]; return o * o; };
    auto epi = [&](int i, double s1, double s2) {
        P.X.btil[i] = P.b[i] + P.mu * s1;
        if (!(s2 > 0.0)) { bad += 1.0; P.V.jinv[i] = T(1); }
        else P.V.jinv[i] = (T)(1.0 / s2);
    };
    sell_rows2(P.A, g1, g2, epi);
    const double v[1] = {bad};
    const int op[1] = {0};
    block_partials<1>(v, op, P.partials);
}

// Start of the projection solve: w <- w + theta (w - w_prev) and, since
// q = A_hat' w is linear in w while O is fixed, q <- q + theta (q - q_prev)
// exactly, with no matrix pass (theta = 0: the previous w, a plain warm
// start).  The outer iteration converges linearly, so consecutive w follow a
// near-geometric sequence and the extrapolated start leaves the correction
// solve a smaller residual.  Returns the q to use; saves the current pair
// when the setting is on (save).
__device__ __forceinline__ double extrap_q(const Outer& X, int j, double theta, bool save) {
    const double q = X.q[j];
    if (theta == 0.0) {
        if (save) X.qp[j] = q;
        return q;
    }
    const double qn = fma(theta, q - X.qp[j], q);
    X.qp[j] = q;
    X.q[j] = qn;
    return qn;
}

// Step 17: p = abs_K(s); g = O (p + q) for the warm-started right-hand side
// (theta: see extrap_q).
// Lorentz cone (v1, vbar), t = ||vbar||: inside (t <= v1) abs = v; polar
// (t <= -v1) abs = -v; otherwise abs = (t, (v1/t) vbar), which is 2 proj - v
// for proj = ((v1 + t)/2)(1, vbar/t).
template <typename T>
__device__ __noinline__ void phase_abs(const IterParams<T>& P, double theta) {
    const Outer& X = P.X;
    const bool save = P.extrap != 0.0;                  // the setting is on: keep the pairs
    if (save)
        for (int i = global_tid(); i < P.m; i += global_threads()) {
            const double w = X.w[i];
            if (theta != 0.0) X.w[i] = fma(theta, w - X.wp[i], w);
            X.wp[i] = w;
        }
    if (P.admm) {                                       // ADMM form: the projection acts on s itself
        for (int j = global_tid(); j < P.n; j += global_threads()) {
            const double pj = X.s[j];
            X.p[j] = pj;
            X.g[j] = X.O[j] * (pj + extrap_q(X, j, theta, save));
        }
        return;
    }
    for (int j = global_tid(); j < P.n_orth; j += global_threads()) {
        const double pj = fabs(X.s[j]);
        X.p[j] = pj;
        X.g[j] = X.O[j] * (pj + extrap_q(X, j, theta, save));
    }
    const int lane = threadIdx.x & 31;
    for (int cI = global_warp(); cI < P.n_soc; cI += global_warps()) {
        const int a = __ldg(P.soc_off + cI), e = __ldg(P.soc_off + cI + 1);
        double ss = 0.0;
        for (int j = a + 1 + lane; j < e; j += 32) ss = fma(X.s[j], X.s[j], ss);
        ss = warp_sum(ss);
        const double t = sqrt(ss);
        const double v1 = X.s[a];
        double ftail, head;
        if (t <= v1) { ftail = 1.0; head = v1; }
        else if (t <= -v1) { ftail = -1.0; head = -v1; }
        else { ftail = v1 / t; head = t; }
        const double Oc = X.O[a];
        for (int j = a + lane; j < e; j += 32) {
            const double pj = (j == a) ? head : ftail * X.s[j];
            X.p[j] = pj;
            X.g[j] = Oc * (pj + extrap_q(X, j, theta, save));
        }
    }
}

// FP64 residual of the projection system r0 = b_tilde - A g (g = O(p + q),
// i.e. b_tilde - A_hat p - M w); the correction CG starts from it:
// r = r0, u = J^{-1} r.  Partial gamma = r'u.
template <typename T>
__device__ __forceinline__ void rhs_epi(const IterParams<T>& P, int i, double sum, double& gam) {
    const T r = (T)(P.X.btil[i] - sum);
    const T u = P.V.jinv[i] * r;
    P.V.r[i] = r;
    P.V.u[i] = u;
    gam += (double)r * (double)u;
}

template <typename T>
__device__ __noinline__ void phase_rhs(const IterParams<T>& P) {
    double gam = 0.0;
    const double* g = P.X.g;
    auto gather = [g](int j) { return g[j]; };
    auto epi = [&](int i, double sum) { rhs_epi(P, i, sum, gam); };
    sell_rows<double>(P.A, gather, epi);
    const double v[1] = {gam};
    const int op[1] = {0};
    block_partials<1>(v, op, P.partials);
}

// FP32 outer products on the L2-gather layout (a segment that need only reach
// a polish level): the projection residual from FP32 values and g rounded to
// FP32, summed in FP32.
template <typename T>
__device__ __noinline__ void phase_rhs_f32(const IterParams<T>& P) {
    double gam = 0.0;
    const double* g = P.X.g;
    auto gather = [g](int j) { return (float)g[j]; };
    auto epi = [&](int i, float sum) { rhs_epi(P, i, (double)sum, gam); };
    sell_rows<float>(P.A, gather, epi);
    const double v[1] = {gam};
    const int op[1] = {0};
    block_partials<1>(v, op, P.partials);
}

// FP32 outer passes: the product A g of the projection residual as a
// column-blocked FP32 pass (g rounded to FP32 as it is staged) ...
template <typename T>
__device__ __noinline__ void phase_rhs_cb(const IterParams<T>& P) {
    cb_pass(P.Acb, P.X.g, &P.ctl->err);
}
// ... and the residual from its partial sums: r0 = b_tilde - A g.
template <typename T>
__device__ __noinline__ void phase_rhs_comb(const IterParams<T>& P) {
    double gam = 0.0;
    cb_combine(P.Acb, &P.ctl->err, [&](int i, float sum) { rhs_epi(P, i, (double)sum, gam); });
    const double v[1] = {gam};
    const int op[1] = {0};
    block_partials<1>(v, op, P.partials);
}

// CG, first half of M u: t = O^2 (A' u) over the rows of A'.
template <typename T>
__device__ __noinline__ void phase_cg_At(const IterParams<T>& P) {
    const T* u = P.V.u;
    auto gather = [u](int i) { return u[i]; };
    auto epi = [&](int j, T sum) { P.V.t[j] = P.V.O2[j] * sum; };
    sell_rows<T>(P.AT, gather, epi);
}

// CG, second half: au = A t (= M u); partial delta = au'u.
template <typename T>
__device__ __noinline__ void phase_cg_A(const IterParams<T>& P) {
    double delta = 0.0;
    const T* t = P.V.t;
    auto gather = [t](int j) { return t[j]; };
    auto epi = [&](int i, T sum) {
        P.V.au[i] = sum;
        delta += (double)sum * (double)P.V.u[i];
    };
    sell_rows<T>(P.A, gather, epi);
    const double v[1] = {delta};
    const int op[1] = {0};
    block_partials<1>(v, op, P.partials);
}

// Column-blocked CG, first half of M u: the partial sums of A'u ...
template <typename T>
__device__ __noinline__ void phase_cg_At_cb(const IterParams<T>& P) {
    cb_pass(P.ATcb, P.V.u, &P.ctl->err);
}
// ... combined: v = A'u, t = O^2 v, and the partial of u'Mu = sum O^2 v^2
// (= ||A_hat'u||^2, the delta of the CG step, known before the A pass).
template <typename T>
__device__ __noinline__ void phase_cg_tcomb(const IterParams<T>& P) {
    double delta = 0.0;
    cb_combine(P.ATcb, &P.ctl->err, [&](int j, float sum) {
        const T v = (T)sum;
        const T t = P.V.O2[j] * v;
        P.V.t[j] = t;
        delta += (double)t * (double)v;
    });
    const double v[1] = {delta};
    const int op[1] = {0};
    block_partials<1>(v, op, P.partials);
}
// Column-blocked CG, second half: the partial sums of A t (= M u), combined
// in the vector step.
template <typename T>
__device__ __noinline__ void phase_cg_A_cb(const IterParams<T>& P) {
    cb_pass(P.Acb, P.V.t, &P.ctl->err);
}

// Chronopoulos-Gear vector step: p = u + beta p, sv = au + beta sv,
// w += alpha p (FP64), r -= alpha sv, u = J^{-1} r; partial gamma = r'u.
// au(i) = (M u)_i: stored by the A pass, or the partial sums of the
// column-blocked A pass added in block order.
template <typename T, bool CB>
__device__ __noinline__ void phase_cg_vec(const IterParams<T>& P, double alpha, T beta) {
    double gam = 0.0;
    const Inner<T>& V = P.V;
    const T a = (T)alpha;
    auto step = [&](int i, T aui) {
        const T pi = fma(beta, V.p[i], V.u[i]);
        const T si = fma(beta, V.sv[i], aui);
        V.p[i] = pi;
        V.sv[i] = si;
        P.X.w[i] += alpha * (double)pi;
        const T r = fma(-a, si, V.r[i]);
        V.r[i] = r;
        const T u = V.jinv[i] * r;
        V.u[i] = u;
        gam += (double)r * (double)u;
    };
    if (CB) cb_combine(P.Acb, &P.ctl->err, [&](int i, float sum) { step(i, (T)sum); });
    else
        for (int i = global_tid(); i < P.m; i += global_threads()) step(i, V.au[i]);
    const double v[1] = {gam};
    const int op[1] = {0};
    block_partials<1>(v, op, P.partials);
}

// q = O (A' w) over the rows of A' (FP64); with update: s <- (s + p)/2 -
// mu c_hat + q (steps 18-19) and, if want_xz, x = O (p + s)/2 and
// z = (p - s)/(2 mu O) (steps 20-21).  Partials ||s_new - s||^2, ||s_new||^2.
// fuse_abs (orthant-only problems, no extrapolation, no rescaling next):
// also step 17 of the next iteration, p = |s_new| and g = O (p + q) with the
// q just formed -- the values phase_abs would compute there.
template <typename T>
__device__ __forceinline__ void update_epi(const IterParams<T>& P, int j, double sum, bool update, bool want_xz,
                                           double& ds2, double& ss2, bool fuse_abs = false) {
    const double Oj = P.X.O[j];
    const double qj = Oj * sum;
    P.X.q[j] = qj;
    if (!update) P.X.g[j] = Oj * (P.X.p[j] + qj);   // right-hand side input of a refinement round
    if (update && P.admm) {
        // ADMM form (Section III-B), as Douglas-Rachford splitting with the two
        // proximal steps in the other order: p = s = zeta, q = A_hat' w with
        // w = M^{-1}(b_tilde - A_hat zeta), so zeta - mu c_hat + q is the
        // proximal point of g (x2) and a = 2 x2 - zeta its reflection;
        // zeta <- (zeta + abs_K(a))/2, x1 = proj_K(a) = (a + abs_K(a))/2 and
        // z = (abs_K(a) - a)/(2 mu), scaled back by O.  Lorentz-cone
        // coordinates keep a in p for phase_admm_soc.
        const double so = P.X.s[j];
        const double a = (so - 2.0 * P.mu * P.X.chat[j]) + 2.0 * qj;
        if (j >= P.n_orth) {
            P.X.p[j] = a;
            return;
        }
        const double aa = fabs(a);
        const double sj = 0.5 * (so + aa);
        P.X.s[j] = sj;
        ds2 += (sj - so) * (sj - so);
        ss2 += sj * sj;
        if (want_xz) {
            P.x[j] = Oj * (a + aa) * 0.5;
            P.z[j] = (aa - a) / (2.0 * P.mu * Oj);
        }
        return;
    }
    if (update) {
        const double pj = P.X.p[j];
        const double so = P.X.s[j];
        const double sj = (0.5 * (so + pj) - P.mu * P.X.chat[j]) + qj;
        P.X.s[j] = sj;
        ds2 += (sj - so) * (sj - so);
        ss2 += sj * sj;
        if (want_xz) {
            P.x[j] = Oj * (pj + sj) * 0.5;
            P.z[j] = (pj - sj) / (2.0 * P.mu * Oj);
        }
        if (fuse_abs) {
            const double pn = fabs(sj);
            P.X.p[j] = pn;
            P.X.g[j] = Oj * (pn + qj);
        }
    }
}

// Partials of the update: ||s_new - s||^2, ||s_new||^2 and, for a
// time-sliced solve, whether the deadline has passed (one clock read per
// CTA, max-reduced, so every CTA of the team takes the same decision).
__device__ __forceinline__ void update_partials(double ds2, double ss2, bool update, double* partials) {
    const unsigned long long dl = sync_smem().deadline;
    const double over = (update && dl != 0ull && threadIdx.x == 0 && gtimer() > dl) ? 1.0 : 0.0;
    const double v[3] = {ds2, ss2, over};
    const int op[3] = {0, 0, 1};
    block_partials<3>(v, op, partials);
}

template <typename T>
__device__ __noinline__ void phase_update(const IterParams<T>& P, bool update, bool want_xz, bool fuse_abs = false) {
    double ds2 = 0.0, ss2 = 0.0;
    const double* w = P.X.w;
    auto gather = [w](int i) { return w[i]; };
    auto epi = [&](int j, double sum) { update_epi(P, j, sum, update, want_xz, ds2, ss2, fuse_abs); };
    sell_rows<double>(P.AT, gather, epi);
    update_partials(ds2, ss2, update, P.partials);
}

// The update from an FP32 product A'w on the L2-gather layout (see phase_rhs_f32).
template <typename T>
__device__ __noinline__ void phase_update_f32(const IterParams<T>& P, bool want_xz, bool fuse_abs) {
    double ds2 = 0.0, ss2 = 0.0;
    const double* w = P.X.w;
    auto gather = [w](int i) { return (float)w[i]; };
    auto epi = [&](int j, float sum) { update_epi(P, j, (double)sum, true, want_xz, ds2, ss2, fuse_abs); };
    sell_rows<float>(P.AT, gather, epi);
    update_partials(ds2, ss2, true, P.partials);
}

// FP32 outer passes: A'w as a column-blocked FP32 pass (w rounded to FP32 as
// it is staged) ...
template <typename T>
__device__ __noinline__ void phase_update_cb(const IterParams<T>& P) {
    cb_pass(P.ATcb, P.X.w, &P.ctl->err);
}
// ... and the update from its partial sums.
template <typename T>
__device__ __noinline__ void phase_update_comb(const IterParams<T>& P, bool want_xz, bool fuse_abs = false) {
    double ds2 = 0.0, ss2 = 0.0;
    cb_combine(P.ATcb, &P.ctl->err,
               [&](int j, float sum) { update_epi(P, j, (double)sum, true, want_xz, ds2, ss2, fuse_abs); });
    update_partials(ds2, ss2, true, P.partials);
}

// ADMM form, Lorentz cones: abs_K of the reflection a kept in p by
// update_epi (the cone rule of phase_abs), then zeta <- (zeta + abs_K(a))/2,
// x and z as for the orthant.  Partials ||s_new - s||^2, ||s_new||^2 of these
// coordinates.
template <typename T>
__device__ __noinline__ void phase_admm_soc(const IterParams<T>& P, bool want_xz) {
    double ds2 = 0.0, ss2 = 0.0;
    const Outer& X = P.X;
    const int lane = threadIdx.x & 31;
    for (int cI = global_warp(); cI < P.n_soc; cI += global_warps()) {
        const int a0 = __ldg(P.soc_off + cI), e = __ldg(P.soc_off + cI + 1);
        double tt = 0.0;
        for (int j = a0 + 1 + lane; j < e; j += 32) tt = fma(X.p[j], X.p[j], tt);
        tt = warp_sum(tt);
        const double t = sqrt(tt);
        const double v1 = X.p[a0];
        double ftail, head;
        if (t <= v1) { ftail = 1.0; head = v1; }
        else if (t <= -v1) { ftail = -1.0; head = -v1; }
        else { ftail = v1 / t; head = t; }
        const double Oc = X.O[a0];
        for (int j = a0 + lane; j < e; j += 32) {
            const double a = X.p[j];
            const double aa = (j == a0) ? head : ftail * a;
            const double so = X.s[j];
            const double sj = 0.5 * (so + aa);
            X.s[j] = sj;
            ds2 += (sj - so) * (sj - so);
            ss2 += sj * sj;
            if (want_xz) {
                P.x[j] = Oc * (a + aa) * 0.5;
                P.z[j] = (aa - a) / (2.0 * P.mu * Oc);
            }
        }
    }
    const double v[2] = {ds2, ss2};
    const int op[2] = {0, 0};
    block_partials<2>(v, op, P.partials);
}

// FP64 residual partials: ||Ax - b||^2, ||A'y + z - c||^2 (y = w/mu), c'x, b'y,
// dist(x,K)^2, dist(z,K)^2, ||x||^2, ||z||^2.
__device__ __forceinline__ double soc_dist2(double v1, double t) {
    // squared distance from (v1, vbar) with ||vbar|| = t to the Lorentz cone
    if (t <= v1) return 0.0;
    if (t <= -v1) return v1 * v1 + t * t;
    const double d = 0.5 * (t - v1);      // distance = |t - v1| / sqrt 2
    return 2.0 * d * d;
}

template <typename T>
__device__ __noinline__ void phase_kkt(const IterParams<T>& P) {
    double rp = 0.0, rd = 0.0, cx = 0.0, by = 0.0, dx = 0.0, dz = 0.0, xx = 0.0, zz = 0.0;
    const double* x = P.x;
    const double* z = P.z;
    const double* w = P.X.w;
    const double inv_mu = 1.0 / P.mu;
    {
        auto gather = [x](int j) { return x[j]; };
        auto epi = [&](int i, double sum) {
            const double d = sum - P.b[i];
            rp += d * d;
            by += P.b[i] * (w[i] * inv_mu);
        };
        sell_rows<double>(P.A, gather, epi);
    }
    {
        auto gather = [w, inv_mu](int i) { return w[i] * inv_mu; };
        auto epi = [&](int j, double sum) {
            const double d = sum + z[j] - P.c[j];
            rd += d * d;
        };
        sell_rows<double>(P.AT, gather, epi);
    }
    for (int j = global_tid(); j < P.n_orth; j += global_threads()) {
        const double xj = x[j], zj = z[j];
        cx += P.c[j] * xj;
        xx += xj * xj;
        zz += zj * zj;
        if (xj < 0.0) dx += xj * xj;
        if (zj < 0.0) dz += zj * zj;
    }
    const int lane = threadIdx.x & 31;
    for (int cI = global_warp(); cI < P.n_soc; cI += global_warps()) {
        const int a = __ldg(P.soc_off + cI), e = __ldg(P.soc_off + cI + 1);
        double sx = 0.0, sz = 0.0, scx = 0.0;
        for (int j = a + 1 + lane; j < e; j += 32) {
            sx = fma(x[j], x[j], sx);
            sz = fma(z[j], z[j], sz);
            scx = fma(P.c[j], x[j], scx);
        }
        sx = warp_sum(sx);
        sz = warp_sum(sz);
        scx = warp_sum(scx);
        if (lane == 0) {
            const double xa = x[a], za = z[a];
            cx += scx + P.c[a] * xa;
            xx += sx + xa * xa;
            zz += sz + za * za;
            dx += soc_dist2(xa, sqrt(sx));
            dz += soc_dist2(za, sqrt(sz));
        }
    }
    const double v[8] = {rp, rd, cx, by, dx, dz, xx, zz};
    const int op[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    block_partials<8>(v, op, P.partials);
}

// ---------------------------------------------------------------------------
// cached projection operator (small m): M = A_hat A_hat' factored once per
// rescaling, then every projection solve is two dense FP64 products
// ---------------------------------------------------------------------------
//
// The operator of the projection (Algorithm 1 step 2 / Algorithm 2 step 12:
// the pseudoinverse of A_hat through M = A_hat A_hat') changes only when O
// does.  For small m it is cached as the explicit inverse factor
// X = L^{-1} of the Cholesky factorisation M = L L' (FP64), so that the
// correction of every iteration, dw = M^{-1} r0 = X' (X r0), is exact up to
// rounding, like the oracle's dense solve, and costs two triangular matrix-
// vector products with no sequential dependence.
// Storage: M row-major [m x m] (lower triangle used, overwritten by L);
// X column-major (X[c * m + i] = (L^{-1})_{ic}, i >= c).

// M = A O^2 A' (lower triangle), from row i of A and the columns of A it
// touches (rows of A'): M_ik = sum_j O_j^2 a_ij a_kj.  Warp per row i, the
// lanes over the entries of one column j at a time, in a fixed order.
// Entry j of row i of a matrix whose rows are full (every column present,
// in order), from its sliced-ELLPACK image: slice i / (32/g), lane group
// i % (32/g), chunk j / g.
__device__ __forceinline__ double sell_full_entry(const SellMat& A, int i, int j) {
    const int g = A.g, h = 32 / g;
    return __ldg(A.v64 + __ldg(A.sptr + i / h) + 32 * (j / g) + (i % h) * g + (j % g));
}

// M = A O^2 A' for full rows (the dense workloads): 64 x 64 tiles of the lower
// triangle dealt to the team's CTAs, each the sum over j in increasing order
// of 64 x 8 slabs of its two row blocks staged in shared memory (the first
// scaled by O_j^2); thread (ty, tx) of the 32 x 32 threads owns rows
// {ty, ty + 32} and columns {tx, tx + 32} of the tile.  FP64 throughout (the
// FP64 pipe bounds it: about two FP64 multiply-adds per clock per SM here, so
// the slabs stay small and leave L1 its carve-out).
constexpr int kSyrkT = 64, kSyrkK = 8;

template <typename T>
__device__ __noinline__ void phase_dense_syrk(const IterParams<T>& P) {
    __shared__ double Ai[kSyrkT][kSyrkK + 1];
    __shared__ double Ak[kSyrkT][kSyrkK + 1];
    double* M = sync_smem().dM;
    const int m = P.m, n = P.n;
    const int mt = (m + kSyrkT - 1) / kSyrkT;
    const long long ntile = (long long)mt * (mt + 1) / 2;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (long long t = team_rank(); t < ntile; t += team_size()) {
        // lower-triangular tile (bi, bk), bk <= bi, t = bi (bi + 1) / 2 + bk
        int bi = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while ((long long)(bi + 1) * (bi + 2) / 2 <= t) ++bi;
        while ((long long)bi * (bi + 1) / 2 > t) --bi;
        const int bk = (int)(t - (long long)bi * (bi + 1) / 2);
        const int i0 = bi * kSyrkT, k0 = bk * kSyrkT;
        double a00 = 0.0, a01 = 0.0, a10 = 0.0, a11 = 0.0;
        for (int j0 = 0; j0 < n; j0 += kSyrkK) {
            for (int e = threadIdx.x; e < kSyrkT * kSyrkK; e += blockDim.x) {
                const int r = e / kSyrkK, c = e % kSyrkK, j = j0 + c;
                double vi = 0.0, vk = 0.0;
                if (j < n) {
                    const double o = P.X.O[j];
                    if (i0 + r < m) vi = sell_full_entry(P.A, i0 + r, j) * (o * o);
                    if (k0 + r < m) vk = sell_full_entry(P.A, k0 + r, j);
                }
                Ai[r][c] = vi;
                Ak[r][c] = vk;
            }
            __syncthreads();
#pragma unroll 8
            for (int c = 0; c < kSyrkK; ++c) {
                const double x0 = Ai[ty][c], x1 = Ai[ty + 32][c];
                const double y0 = Ak[tx][c], y1 = Ak[tx + 32][c];
                a00 = fma(x0, y0, a00);
                a01 = fma(x0, y1, a01);
                a10 = fma(x1, y0, a10);
                a11 = fma(x1, y1, a11);
            }
            __syncthreads();
        }
        const double acc[2][2] = {{a00, a01}, {a10, a11}};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const int i = i0 + ty + 32 * a, k = k0 + tx + 32 * b;
                if (i < m && k <= i) M[(size_t)i * m + k] = acc[a][b];
            }
    }
}

template <typename T>
__device__ __noinline__ void phase_dense_assemble(const IterParams<T>& P) {
    if (P.full_rows && blockDim.x == 1024) {            // dense rows: tiled product
        phase_dense_syrk(P);
        return;
    }
    double* M = sync_smem().dM;
    const int m = P.m;
    const int lane = threadIdx.x & 31;
    const SellMat& A = P.A;
    const SellMat& AT = P.AT;
    for (int i = global_warp(); i < m; i += global_warps()) {
        double* Mi = M + (size_t)i * m;
        for (int k = lane; k <= i; k += 32) Mi[k] = 0.0;
        __syncwarp();
        const int ga = A.g, ha = 32 / ga;
        const int sl = i / ha, lr = i % ha;
        const int base = __ldg(A.sptr + sl), len = __ldg(A.slen + sl) * ga;
        for (int e = 0; e < len; ++e) {
            const int idx = base + 32 * (e / ga) + lr * ga + (e % ga);
            const double aij = __ldg(A.v64 + idx);
            if (aij == 0.0) continue;                         // padding
            const int j = __ldg(A.col + idx);
            const double Oj = P.X.O[j];
            const double f = aij * Oj * Oj;
            // column j of A = row j of A' (relabelled rows, increasing)
            const int gt = AT.g, ht = 32 / gt;
            const int slt = j / ht, lrt = j % ht;
            const int bt = __ldg(AT.sptr + slt), lt = __ldg(AT.slen + slt) * gt;
            for (int q = lane; q < lt; q += 32) {
                const int it = bt + 32 * (q / gt) + lrt * gt + (q % gt);
                const double akj = __ldg(AT.v64 + it);
                const int k = __ldg(AT.col + it);
                if (akj != 0.0 && k <= i) Mi[k] = fma(f, akj, Mi[k]);
            }
            __syncwarp();
        }
    }
}

// Pivot rule of the factorisation: a pivot below 1e-13 of the row's
// original diagonal (jinv = 1 / diag M) marks row k of A as linearly
// dependent on the rows before it (rank-deficient A): the direction is
// dropped -- the pivot becomes +inf, its column of L is zero, nothing is
// eliminated with it, and row k of L^{-1} is zero.  For a consistent
// right-hand side (b in range(A)) this solves the remaining independent
// equations, which imply the dropped one.  A pivot negative beyond rounding
// or not a number fails the factorisation.
// Blocked right-looking Cholesky: kCholB columns per step and two team
// barriers per step (instead of one per column), so the trailing triangle is
// read and rewritten once per kCholB columns.  The result has the layout of
// the column-by-column version: the pivot d_k on the diagonal (+inf for a
// dependent row), L below it.
//   Step at column k0, block b = min(kCholB, m - k0):
//   1. every CTA factors the diagonal block D = M[k0.., k0..] (b x b) in
//      shared memory, column by column with the pivot rule above, so every
//      CTA takes the same decisions without communicating; CTA 0 writes it
//      back;
//   2. every row i below the block is solved against it (warp per row):
//      L_ik = (M_ik - sum_{t<k} L_it L_kt) s_k with s_k = 1/sqrt(d_k) (0 for
//      a dependent row);
//   -- team barrier --
//   3. the trailing lower triangle is updated by the panel (warp per row i,
//      lanes over the columns j <= i): M_ij -= sum_t L_it L_jt.
//   -- team barrier --
// Returns false (in every thread of the team) only for a pivot that is
// negative beyond rounding or not a number.
constexpr int kCholB = 16;

template <typename T>
__device__ __noinline__ bool dense_chol_panel(double* M, int m, int k0, const T* jinv) {
    __shared__ double D[kCholB][kCholB];
    __shared__ double sc[kCholB];
    __shared__ int bad;
    const int b = min(kCholB, m - k0);
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int r = e / b, c = e % b;
        D[r][c] = r >= c ? __ldcg(M + (size_t)(k0 + r) * m + k0 + c) : 0.0;
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    if (threadIdx.x < 32) {                              // one warp factors the block
        const int lane = threadIdx.x;
        for (int k = 0; k < b; ++k) {
            const double d = D[k][k];
            const double tau = 1e-13 / (double)__ldcg(jinv + k0 + k);
            const bool fail = d != d || d < -1e3 * tau;
            const bool dep = !(d > tau) || d == INFINITY;
            const double s = dep ? 0.0 : 1.0 / sqrt(d);
            __syncwarp();
            if (lane == 0) {
                if (fail) bad = 1;
                sc[k] = s;
                D[k][k] = dep ? INFINITY : d;
            }
            if (lane > k && lane < b) D[lane][k] *= s;  // column k of L in the block
            __syncwarp();
            for (int i = k + 1 + lane; i < b; i += 32)   // rows below: update columns k+1 .. i
                for (int j = k + 1; j <= i; ++j) D[i][j] = fma(-D[i][k], D[j][k], D[i][j]);
            __syncwarp();
        }
    }
    __syncthreads();
    if (bad) return false;                               // CTA-uniform (and team-uniform: same data)
    if (team_rank() == 0)
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
            const int r = e / b, c = e % b;
            if (r >= c) M[(size_t)(k0 + r) * m + k0 + c] = D[r][c];
        }
    // panel rows below the block, warp per row, lane k holds L_ik
    const int lane = threadIdx.x & 31;
    for (int i = k0 + b + global_warp(); i < m; i += global_warps()) {
        double* Mi = M + (size_t)i * m + k0;
        double x = lane < b ? __ldcg(Mi + lane) : 0.0;
        for (int k = 0; k < b; ++k) {
            const double xk = __shfl_sync(0xffffffffu, x, k) * sc[k];   // final L_ik
            if (lane == k) x = xk;
            if (lane > k && lane < b) x = fma(-xk, D[lane][k], x);
        }
        if (lane < b) Mi[lane] = x;
    }
    return true;
}

// Step 3 of the blocked factorisation: M_ij -= sum_t L_it L_jt for
// k0 + b <= j <= i < m, with L the panel just written.
static __device__ __noinline__ void dense_chol_trailing(double* M, int m, int k0) {
    const int b = min(kCholB, m - k0);
    const int lane = threadIdx.x & 31;
    for (int i = k0 + b + global_warp(); i < m; i += global_warps()) {
        const double* Li = M + (size_t)i * m + k0;
        double li[kCholB];
#pragma unroll
        for (int t = 0; t < kCholB; ++t) li[t] = t < b ? __ldcg(Li + t) : 0.0;
        double* Mi = M + (size_t)i * m;
        for (int j = k0 + b + lane; j <= i; j += 32) {
            const double* Lj = M + (size_t)j * m + k0;
            double acc = 0.0;
#pragma unroll
            for (int t = 0; t < kCholB; ++t)
                if (t < b) acc = fma(li[t], __ldcg(Lj + t), acc);
            Mi[j] -= acc;
        }
    }
}

// X = L^{-1} (column-major) by forward substitution, warp per column c:
// x_i = (delta_ic - sum_{c <= t < i} L_it x_t) / L_ii for i >= c, with
// L_ii = sqrt(d_i) from the pivot kept on the diagonal.
template <typename T>
__device__ __noinline__ void phase_dense_inverse(const IterParams<T>& P) {
    const double* M = sync_smem().dM;
    double* X = sync_smem().dX;
    const int m = P.m;
    const int lane = threadIdx.x & 31;
    for (int c = global_warp(); c < m; c += global_warps()) {
        double* Xc = X + (size_t)c * m;
        for (int i = c; i < m; ++i) {
            const double* Li = M + (size_t)i * m;
            double acc = 0.0;
            for (int t = c + lane; t < i; t += 32) acc = fma(__ldcg(Li + t), Xc[t], acc);
            acc = warp_sum(acc);
            const double xi = ((i == c ? 1.0 : 0.0) - acc) / sqrt(__ldcg(Li + i));
            if (lane == 0) Xc[i] = xi;
            __syncwarp();
        }
    }
}

// y = X r0 (r0 = the FP64 residual of the projection system, in V.r), thread
// per row; y is kept in V.p (unused by the dense path).
template <typename T>
__device__ __noinline__ void phase_dense_y(const IterParams<T>& P) {
    const double* X = sync_smem().dX;
    const int m = P.m;
    const T* r = P.V.r;
    for (int i = global_tid(); i < m; i += global_threads()) {
        // four independent partial sums keep four loads of X in flight
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int c = 0;
        for (; c + 3 <= i; c += 4) {
            a0 = fma(__ldcg(X + (size_t)c * m + i), (double)__ldcg(r + c), a0);
            a1 = fma(__ldcg(X + (size_t)(c + 1) * m + i), (double)__ldcg(r + c + 1), a1);
            a2 = fma(__ldcg(X + (size_t)(c + 2) * m + i), (double)__ldcg(r + c + 2), a2);
            a3 = fma(__ldcg(X + (size_t)(c + 3) * m + i), (double)__ldcg(r + c + 3), a3);
        }
        for (; c <= i; ++c) a0 = fma(__ldcg(X + (size_t)c * m + i), (double)__ldcg(r + c), a0);
        P.V.p[i] = (T)((a0 + a1) + (a2 + a3));
    }
}

// w += X' y: warp per column c, x_c = sum_{i >= c} X_ic y_i.
template <typename T>
__device__ __noinline__ void phase_dense_x(const IterParams<T>& P) {
    const double* X = sync_smem().dX;
    const int m = P.m;
    const int lane = threadIdx.x & 31;
    const T* y = P.V.p;
    for (int c = global_warp(); c < m; c += global_warps()) {
        const double* Xc = X + (size_t)c * m;
        double a0 = 0.0, a1 = 0.0;
        int i = c + lane;
        for (; i + 32 < m; i += 64) {
            a0 = fma(__ldcg(Xc + i), (double)__ldcg(y + i), a0);
            a1 = fma(__ldcg(Xc + i + 32), (double)__ldcg(y + i + 32), a1);
        }
        if (i < m) a0 = fma(__ldcg(Xc + i), (double)__ldcg(y + i), a0);
        const double acc = warp_sum(a0 + a1);
        if (lane == 0) P.X.w[c] += acc;
    }
}

// ---------------------------------------------------------------------------
// LP crossover polish (FP64; the entry point is acs_polish).  Support
// B = {j : x_j > z_j}; O holds the indicator of B, so that the projection-
// solve phases work with M = A O^2 A' = A_B A_B' unchanged:
//   x~ = O (p + q), p = O x, q = O A'w, w solving M w = b - A O p (refinement
//        rounds of phase_rhs / CG / phase_update from w = 0);
//   y~ = y + d, d solving M d = A O (O z_y), z_y = c - A'y (the same rounds
//        with b_tilde = 0 and p = -O z_y), a Jacobi-preconditioned CG from
//        zero: the least change of y in the metric J = diag(M);
//   z~ = c - A'y~.
// ---------------------------------------------------------------------------

constexpr int kPolishWindow = 100;   // CG iterations over which the residual must halve

struct PolishOut {
    double* px;      // [n] polished x
    double* pw;      // [m] on entry the iterate's w = mu y; on exit mu y~
                     //     (the solves accumulate in P.X.w, a scratch vector)
    double* pz;      // [n] polished z
    double* res;     // [6] residuals of the polished point (as ctl->res) ...
    double* info;    // [5] |B|, CG iterations (dense: corrections) of the x and y
                     //     solves, 1 = completed, 1 = the factored M was used
};

// O = indicator of B, p = O x, q = 0, g = O (p + q), w = 0, and the count |B|.
static __device__ __noinline__ void phase_polish_init(const IterParams<double>& P, float* O2_32) {
    double nb = 0.0;
    for (int j = global_tid(); j < P.n; j += global_threads()) {
        const double o = P.x[j] > P.z[j] ? 1.0 : 0.0;
        nb += o;
        P.X.O[j] = o;
        P.V.O2[j] = o;
        if (O2_32) O2_32[j] = (float)o;
        const double pj = o * P.x[j];
        P.X.p[j] = pj;
        P.X.q[j] = 0.0;
        P.X.g[j] = pj;
        P.X.chat[j] = fabs(pj);                       // magnitudes behind the residual's rounding
    }
    for (int i = global_tid(); i < P.m; i += global_threads()) P.X.w[i] = 0.0;
    const double v[1] = {nb};
    const int op[1] = {0};
    block_partials<1>(v, op, P.partials);
}

// b_tilde = b and J^{-1} = 1 / diag(A_B A_B') (1 on rows without an entry in B).
template <typename T>
__device__ __noinline__ void phase_polish_jacobi(const IterParams<T>& P) {
    const double* O = P.X.O;
    auto g1 = [](int) { return 0.0; };
    auto g2 = [O](int j) { return O[j]; };
    auto epi = [&](int i, double, double s2) {
        P.X.btil[i] = P.b[i];
        P.V.jinv[i] = (T)(s2 > 0.0 ? 1.0 / s2 : 1.0);
    };
    sell_rows2(P.A, g1, g2, epi);
}

// After the x solve: px = g (= x~); z_y = c - A'(w_iter / mu) into pz; the
// y solve's start p = -O z_y, q = 0, g = O p, w = 0, b_tilde = 0.
static __device__ __noinline__ void phase_polish_ystart(const IterParams<double>& P, const PolishOut& out) {
    const double* pw = out.pw;
    const double inv_mu = 1.0 / P.mu;
    auto gather = [pw, inv_mu](int i) { return pw[i] * inv_mu; };
    auto epi = [&](int j, double sum) {
        const double o = P.X.O[j];
        out.px[j] = P.X.g[j];
        const double zj = P.c[j] - sum;
        out.pz[j] = zj;
        const double pj = -o * zj;
        P.X.p[j] = pj;
        P.X.q[j] = 0.0;
        P.X.g[j] = o * pj;
        P.X.chat[j] = o * (fabs(P.c[j]) + fabs(sum));
    };
    sell_rows<double>(P.AT, gather, epi);
    for (int i = global_tid(); i < P.m; i += global_threads()) {
        P.X.w[i] = 0.0;
        P.X.btil[i] = 0.0;
    }
}

// z~ = c - A'(pw / mu).
static __device__ __noinline__ void phase_polish_z(const IterParams<double>& P, const PolishOut& out) {
    const double* pw = out.pw;
    const double inv_mu = 1.0 / P.mu;
    auto gather = [pw, inv_mu](int i) { return pw[i] * inv_mu; };
    auto epi = [&](int j, double sum) { out.pz[j] = P.c[j] - sum; };
    sell_rows<double>(P.AT, gather, epi);
}

// Products over the rows of A' restricted to the support: a lane whose row
// j has O_j = 0 issues no loads (its result is 0), so a pass costs about the
// support's share of the matrix stream and gathers.  Plain loop (one chunk
// at a time); FP64 values.
template <typename T, typename Epi, typename Gather>
__device__ __forceinline__ void sell_rows_active(const SellMat& M, const double* __restrict__ O, Gather gather,
                                                 Epi epi) {
    const int lane = threadIdx.x & 31;
    const int g = M.g, h = 32 / g;
    const T* __restrict__ val = sell_vals<T>(M);
    for (int sl = global_warp(); sl < M.nslices; sl += global_warps()) {
        const int row = sl * h + lane / g;
        const bool act = row < M.nrows && O[row] != 0.0;
        const int len = __ldg(M.slen + sl);
        int idx = __ldg(M.sptr + sl) + lane;
        T acc = T(0);
        if (act)
            for (int k = 0; k < len; ++k, idx += 32) acc = fma(ld_stream(val + idx), gather(ld_stream(M.col + idx)), acc);
        for (int o = g / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((lane & (g - 1)) == 0 && row < M.nrows) epi(row, act ? acc : T(0));
    }
}

// The polish's CG half-step t = O^2 A'u and its q refresh q = O A'w,
// g = O (p + q), on the support's rows only (O is the support's indicator).
template <typename T>
__device__ __noinline__ void phase_polish_cg_At(const IterParams<T>& P) {
    const T* u = P.V.u;
    sell_rows_active<T>(P.AT, P.X.O, [u](int i) { return u[i]; },
                        [&](int j, T sum) { P.V.t[j] = P.V.O2[j] * sum; });
}
static __device__ __noinline__ void phase_polish_q(const IterParams<double>& P) {
    const double* w = P.X.w;
    sell_rows_active<double>(P.AT, P.X.O, [w](int i) { return w[i]; }, [&](int j, double sum) {
        const double o = P.X.O[j];
        const double q = o * sum;
        P.X.q[j] = q;
        P.X.g[j] = o * (P.X.p[j] + q);
    });
}

// The projection residual r0 = b_tilde - A g with its rounding floor: the
// partials are r0' J^{-1} r0 and sum_i J^{-1}_i (b_tilde_i^2 + sum_j A_ij^2
// h_j^2), h (in c_hat) the magnitudes whose rounding the residual carries
// (|x_B| for the x solve, |c_B| + |A_B'y| for the y solve).
template <typename T>
__device__ __noinline__ void phase_polish_rhs(const IterParams<T>& P) {
    double gam = 0.0, fl = 0.0;
    const double* g = P.X.g;
    const double* h = P.X.chat;
    auto g1 = [g](int j) { return g[j]; };
    auto g2 = [h](int j) { return h[j] * h[j]; };
    auto epi = [&](int i, double sum, double s2) {
        rhs_epi(P, i, sum, gam);
        const double bt = P.X.btil[i];
        fl += P.V.jinv[i] * (bt * bt + s2);
    };
    sell_rows2(P.A, g1, g2, epi);
    const double v[2] = {gam, fl};
    const int op[2] = {0, 0};
    block_partials<2>(v, op, P.partials);
}

// M w = b_tilde - A g by FP64 refinement rounds (FP64 residual, Jacobi-PCG
// correction to 1e-13 of the round's residual, the residual's rounding
// floor 64 eps (sum J^{-1}(b_tilde^2 + (Ag)^2))^{1/2} with eps = 2^-52, the
// target rel times the first residual, or cg_max iterations), until the
// residual is at that floor or target, stops falling tenfold a round, or
// `rounds` rounds have run; then q = O A'w and g = O (p + q) for the final w.
// (Residuals in the J^{-1}-norm.)
// When |B| < m, M is singular and the rounding of b_tilde - A g leaves a
// part outside range(M) that no correction removes: the floor ends the
// solve there instead of letting CG drift on it.  Returns false on a failed
// barrier or a non-finite residual.
template <typename T>
__device__ bool polish_solve(const IterParams<double>& P, const IterParams<T>& PT, int rounds, double rel,
                             bool dense, long long& cg_total) {
    double gam_last = INFINITY, target = 0.0;
    for (int round = 0; round < rounds; ++round) {
        if (round > 0) {
            phase_polish_q(P);
            if (!grid_sync(&P.ctl->err)) return false;
        }
        phase_polish_rhs(PT);
        if (!grid_sync(&P.ctl->err)) return false;
        double gam, floor_r;
        {
            double t2[2];
            const int op[2] = {0, 0};
            grid_combine<2>(P.partials, op, t2);
            gam = t2[0];
            floor_r = 64.0 * 0x1p-52 * sqrt(fmax(t2[1], 0.0));
        }
        if (!isfinite(gam) || !isfinite(floor_r)) return false;
        if (round == 0) target = rel * sqrt(fmax(gam, 0.0));
        floor_r = fmax(floor_r, target);
        if (!(sqrt(fmax(gam, 0.0)) > floor_r) || (round > 0 && gam > 0.01 * gam_last)) break;
        gam_last = gam;
        if (sizeof(T) == 8 && dense) {                 // one exact correction: dw = X'(X r0)
            phase_dense_y(P);
            if (!grid_sync(&P.ctl->err)) return false;
            phase_dense_x(P);
            if (!grid_sync(&P.ctl->err)) return false;
            ++cg_total;
            continue;
        }
        // an FP32 correction goes down to ~1e-5 of its round's residual; the
        // next round's FP64 residual refines it
        const double thr = fmax((sizeof(T) == 4 ? 1e-5 : 1e-13) * sqrt(gam), floor_r);
        double gam_prev = 1.0, alpha_prev = 1.0;
        // and, should the floor underestimate that part, the round ends
        // when the smallest residual so far has not halved in kPolishWindow
        // iterations
        double best = gam, best_ref = gam;
        int k = 0;
        while (sqrt(fmax(gam, 0.0)) > thr && k < P.cg_max) {
            double dl[1];
            const int op1[1] = {0};
            phase_polish_cg_At(PT);
            if (!grid_sync(&P.ctl->err)) return false;
            phase_cg_A(PT);
            if (!grid_sync(&P.ctl->err)) return false;
            grid_combine<1>(P.partials, op1, dl);
            const double beta = (k == 0) ? 0.0 : gam / gam_prev;
            const double denom = dl[0] - ((k == 0) ? 0.0 : beta * gam / alpha_prev);
            if (!(denom > 0.0)) break;                  // attainable accuracy reached
            const double alpha = gam / denom;
            phase_cg_vec<T, false>(PT, alpha, (T)beta);
            if (!grid_sync(&P.ctl->err)) return false;
            double gn[1];
            grid_combine<1>(P.partials, op1, gn);
            gam_prev = gam;
            alpha_prev = alpha;
            gam = gn[0];
            ++k;
            if (!isfinite(gam)) return false;
            best = fmin(best, gam);
            if (k % kPolishWindow == 0) {
                if (best > 0.5 * best_ref) break;
                best_ref = best;
            }
        }
        cg_total += k;
    }
    phase_polish_q(P);
    return grid_sync(&P.ctl->err);
}

// The whole polish; Q is P with x = px, z = pz, w = pw (its KKT residuals).
// fp32: the corrections by FP32 CG on P32 (the same state, FP32 CG vectors
// and values), refined by the FP64 residual of every round.
static __device__ __noinline__ void polish_loop(const IterParams<double>& P, const IterParams<float>& P32,
                                         const IterParams<double>& Q, const PolishOut& out, int rounds,
                                         double rel, bool fp32) {
    const bool owner = blockIdx.x == 0 && threadIdx.x == 0;
    long long cg_x = 0, cg_y = 0;
    double nb[1] = {0.0};
    bool ok = false;
    // with scratch for it, M = A_B A_B' is factored once (the cached
    // operator's phases with O the indicator of B) and both solves apply
    // L^{-1}; a failed factorisation falls back to CG
    bool dense = sync_smem().dM != nullptr;
    double used_dense = 0.0;
    do {
        if (dense) fp32 = false;
        phase_polish_init(P, fp32 ? P32.V.O2 : nullptr);
        if (!grid_sync(&P.ctl->err)) break;
        {
            const int op[1] = {0};
            grid_combine<1>(P.partials, op, nb);
        }
        if (fp32) phase_polish_jacobi(P32);
        else phase_polish_jacobi(P);
        if (!grid_sync(&P.ctl->err)) break;
        if (dense) {
            phase_dense_assemble(P);
            if (!grid_sync(&P.ctl->err)) break;
            bool fine = true;
            for (int k0 = 0; k0 < P.m; k0 += kCholB) {
                if (!dense_chol_panel(sync_smem().dM, P.m, k0, P.V.jinv)) dense = false;
                if (!(fine = grid_sync(&P.ctl->err))) break;
                if (!dense) break;
                dense_chol_trailing(sync_smem().dM, P.m, k0);
                if (!(fine = grid_sync(&P.ctl->err))) break;
            }
            if (!fine) break;
            if (dense) {
                phase_dense_inverse(P);
                if (!grid_sync(&P.ctl->err)) break;
                used_dense = 1.0;
            }
        }
        if (!(fp32 ? polish_solve(P, P32, rounds, rel, false, cg_x)
                   : polish_solve(P, P, rounds, rel, dense, cg_x))) break;     // x~ = g
        phase_polish_ystart(P, out);
        if (!grid_sync(&P.ctl->err)) break;
        if (!(fp32 ? polish_solve(P, P32, rounds, rel, false, cg_y)
                   : polish_solve(P, P, rounds, rel, dense, cg_y))) break;     // d = w
        for (int i = global_tid(); i < P.m; i += global_threads()) out.pw[i] += P.mu * P.X.w[i];
        if (!grid_sync(&P.ctl->err)) break;
        phase_polish_z(P, out);
        if (!grid_sync(&P.ctl->err)) break;
        phase_kkt(Q);
        if (!grid_sync(&P.ctl->err)) break;
        double r8[8];
        const int op[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        grid_combine<8>(P.partials, op, r8);
        if (owner) {
            out.res[0] = sqrt(r8[0]) / (1.0 + P.bnorm);
            out.res[1] = sqrt(r8[1]) / (1.0 + P.cnorm);
            out.res[2] = fabs(r8[2] - r8[3]) / (1.0 + fabs(r8[2]) + fabs(r8[3]));
            out.res[3] = fmax(sqrt(r8[4]), sqrt(r8[5])) / (1.0 + fmax(sqrt(r8[6]), sqrt(r8[7])));
            out.res[4] = r8[2];
            out.res[5] = r8[3];
        }
        ok = true;
    } while (false);
    if (owner) {
        out.info[0] = nb[0];
        out.info[1] = (double)cg_x;
        out.info[2] = (double)cg_y;
        out.info[3] = ok ? 1.0 : 0.0;
        out.info[4] = used_dense;
        P.ctl->bar_gen = sync_smem().gen;
    }
}

// ---------------------------------------------------------------------------
// the solve loop
// ---------------------------------------------------------------------------

// Algorithm 2 from the state in P (fresh, resumed, or handed over by an FP32
// loop when status0 = ST_SWITCH) until the KKT test passes, the iteration
// limit is reached, or the FP32 correction solve hands over.  Run by every
// thread of every CTA of the problem's team (team_set first); the team's
// barrier generation must be current in shared memory (sync_init).  Returns
// the loop's status, the same in every thread of the team; the team's rank-0
// CTA writes it, the residuals and the counters to P.ctl.
template <typename T>
__device__ __noinline__ int solve_loop(const IterParams<T>& P, int status0) {
    Control* ctl = P.ctl;
    // per-phase time record, kept by thread 0 of the team's CTA 0 in shared memory
    __shared__ unsigned long long s_ph_ns[PH_COUNT], s_ph_n[PH_COUNT], s_last;
    const bool clock_owner = team_rank() == 0 && threadIdx.x == 0;
    if (clock_owner) {
        for (int i = 0; i < PH_COUNT; ++i) { s_ph_ns[i] = 0; s_ph_n[i] = 0; }
        s_last = gtimer();
    }

    // state left by the reset or by an earlier loop (written by the team's
    // rank 0 before a barrier): read past L1
    int l = __ldcg(&ctl->l);
    bool refresh = P.refresh != 0 || status0 == ST_SWITCH;
    int status = ST_RUNNING;
    long long cg_total = 0;
    long long nA = 0, nAT = 0, nA64 = 0, nAT64 = 0, ncond = 0, nchk = 0, nA32 = 0, nAT32 = 0;
    // FP32 loop of the single-problem launch: column-blocked CG passes, and
    // FP32 outer passes while P.outer32 is on (until ctl->outer32_end is set)
    const bool cbcg = sizeof(T) == 4 && P.Acb.nblocks > 0 && P.ATcb.nblocks > 0;
    int outer32_end = __ldcg(&ctl->outer32_end);
    bool outer32 = cbcg && P.outer32 != 0 && outer32_end == 0;
    double best_mx = INFINITY;
    int flat_checks = 0;
    double res[6];
    for (int i = 0; i < 6; ++i) res[i] = __ldcg(&ctl->res[i]);
    double ds = __ldcg(&ctl->ds), snorm = __ldcg(&ctl->snorm);
    double eta = __ldcg(&ctl->eta);
    bool ok = true;
    // cached projection operator (FP64 loops only); a factorisation that fails
    // (M singular: rank-deficient A) hands this solve to the CG projection
    // P.dense == 2: start with CG and switch to the cached operator once the
    // CG iterations since the last rescaling exceed P.switch_budget, the cost
    // of one factorisation counted in CG iterations (rent until the price of
    // buying is spent): a member that finishes soon after a rescaling never
    // pays for a factorisation, one whose M is too ill-conditioned for
    // Jacobi-CG pays at most twice the better of the two.  An FP32 loop hands
    // over to the FP64 loop for that, marking the switch in ctl->dense_on; a
    // hand-over for FP32 precision alone continues with FP64 CG under the
    // same rule.
    const bool have_scratch = sync_smem().dM != nullptr;
    bool dense = sizeof(T) == 8 && have_scratch &&
                 (P.dense == 1 || (P.dense == 2 && __ldcg(&ctl->dense_on) != 0));
    bool want_dense = false;                            // FP32 loop: hand over for the switch
    const bool may_switch = P.dense == 2 && (sizeof(T) == 4 ? P.switch_ok != 0 : have_scratch);
    bool dense_failed = __ldcg(&ctl->dense_failed) != 0;
    // a factor held in the problem's own scratch stays valid across a pause
    // (O changes only at rescalings, which refactor)
    bool factor_ok = __ldcg(&ctl->factor_ok) != 0;
    bool factor_kept = P.own_scratch != 0 && factor_ok;
    bool over = false;                                  // deadline of a time-sliced solve passed
    bool extrap_ok = __ldcg(&ctl->extrap_ok) != 0;
    long long win_cg = __ldcg(&ctl->win_cg);
    int win_it = __ldcg(&ctl->win_it);
    long long ndense = 0, nfactor = 0;
    bool abs_fused = false;                             // p, g of the next iteration already formed
    // FP32 outer products on the L2-gather layout (FP32 loop, a segment that
    // ends at a polish level)
    const bool outer32_l2 = sizeof(T) == 4 && P.outer32_l2 != 0 && !cbcg && P.A.v32 && P.AT.v32;

// grid barrier that ends phase `ph`; leaves the enclosing loop on error
#define ACS_SYNC(ph)                                                      \
    {                                                                     \
        if (!(ok = grid_sync(&ctl->err))) break;                                \
        if (clock_owner) {                                                \
            const unsigned long long t_ = gtimer();                       \
            s_ph_ns[ph] += t_ - s_last;                                   \
            s_ph_n[ph] += 1;                                              \
            s_last = t_;                                                  \
        }                                                                 \
    }

    while (ok) {
        if (l >= P.max_iter) { status = ACS_MAX_ITER; break; }
        const int lnext = l + 1;
        const bool cond = (lnext == 1) || in_schedule(P, lnext);
        if (cond) {                                     // a new scaling: a new rental
            win_cg = 0;
            win_it = 0;
        }
        if (may_switch && !dense && !dense_failed && win_cg > P.switch_budget) {
            if (sizeof(T) == 4) {
                want_dense = true;
                status = ST_SWITCH;
                break;
            }
            dense = true;
            refresh = true;                                     // factor at this iteration
        }
        if (cond) {                                             // steps 5-14
            phase_cond_o(P);
            ACS_SYNC(PH_COND_O);
            double mm[3];
            const int op[3] = {1, 1, 0};
            grid_combine<3>(P.partials, op, mm);
            CondRange R;
            R.any = mm[2] > 0.0;                               // some o finite and positive
            R.lmax = mm[0];
            R.lmin = -mm[1];
            const double spread = R.lmax - R.lmin;             // log max o - log min o
            if (!R.any) R.alpha = 0.0;
            else if (!(spread > 0.0)) R.alpha = 1.0;
            else R.alpha = fmin(1.0, P.t_cond / spread);
            phase_cond_apply(P, R, true, true);
            ACS_SYNC(PH_COND_APPLY);
            ++ncond;
        } else if (refresh) {
            phase_cond_apply(P, CondRange{0.0, 0.0, 0.0, false}, false, false);
            ACS_SYNC(PH_COND_APPLY);
        }
        if (cond || refresh) {
            phase_btilde(P);
            ++nA64;
            ACS_SYNC(PH_BTILDE);
            double bb[1];
            const int op[1] = {0};
            grid_combine<1>(P.partials, op, bb);
            if (bb[0] > 0.0) { atomicCAS(&ctl->err, 0, ACS_ERR_FACTOR); ok = false; break; }
            if (cond) factor_ok = false;                    // O changed: the factor is stale
            if (dense && factor_kept && !cond) {
                factor_kept = false;                        // resumed: the cached factor is current
            } else if (dense) {
                factor_kept = false;
                factor_ok = false;
                phase_dense_assemble(P);
                ACS_SYNC(PH_DENSE_ASSEMBLE);
                for (int k0 = 0; k0 < P.m && dense; k0 += kCholB) {
                    if (!dense_chol_panel(sync_smem().dM, P.m, k0, P.V.jinv)) {
                        dense = false;
                        dense_failed = true;
                    }
                    ACS_SYNC(PH_DENSE_FACTOR);
                    if (!dense) break;
                    dense_chol_trailing(sync_smem().dM, P.m, k0);
                    ACS_SYNC(PH_DENSE_FACTOR);
                }
                if (!ok) break;
                if (dense) {
                    phase_dense_inverse(P);
                    ACS_SYNC(PH_DENSE_INVERSE);
                    ++nfactor;
                    factor_ok = true;
                }
            }
            phase_update(P, false, false);                      // q = A_hat' w for the warm start
            ++nAT64;
            ACS_SYNC(PH_QREFRESH);
            refresh = false;
        }

        // extrapolated start, valid once the previous iteration ran in the
        // same scaling (not on an iteration that rescales); skipped when the
        // previous update already formed p and g (and nothing changed O or g since)
        if (!(abs_fused && !cond && !refresh)) {
            phase_abs(P, (extrap_ok && !cond) ? P.extrap : 0.0);   // step 17
            ACS_SYNC(PH_ABS);
        }
        abs_fused = false;
        extrap_ok = true;
        // Projection solve: `refine` rounds of (FP64 residual, correction CG in
        // precision T); a round after the first refreshes q = A_hat' w first.
        bool trouble = false;                                   // FP32 solve cannot keep up
        if (dense) {
            // one exact correction: dw = X'(X r0)
            phase_rhs(P);
            ++nA64;
            ACS_SYNC(PH_RHS);
            phase_dense_y(P);
            ACS_SYNC(PH_DENSE_SOLVE);
            phase_dense_x(P);
            ACS_SYNC(PH_DENSE_SOLVE);
            ++ndense;
        }
        for (int round = 0; round < (dense ? 0 : P.refine); ++round) {
            if (round > 0) {
                phase_update(P, false, false);
                ++nAT64;
                ACS_SYNC(PH_QREFRESH);
            }
            if (outer32) {                                      // r0 from an FP32 product
                phase_rhs_cb(P);
                ++nA32;
                ACS_SYNC(PH_RHS);
                phase_rhs_comb(P);
                ACS_SYNC(PH_RHS_COMB);
            } else if (outer32_l2) {
                phase_rhs_f32(P);                               // r0 from an FP32 product
                ++nA32;
                ACS_SYNC(PH_RHS);
            } else {
                phase_rhs(P);                                   // r0 in FP64
                ++nA64;
                ACS_SYNC(PH_RHS);
            }
            double gam;
            {
                double t1[1];
                const int op[1] = {0};
                grid_combine<1>(P.partials, op, t1);
                gam = t1[0];
            }
            if (!isfinite(gam)) { status = ACS_ERR_NUMERICAL; break; }
            // the step-relative rule needs a previous step in the same scaling;
            // on the first iteration and whenever O changes only the floors apply
            const double rel = (isfinite(ds) && !cond && round == 0) ? eta * ds : 0.0;
            const double thr = fmax(fmax(rel, P.cg_tol * snorm), P.cg_relfloor * sqrt(fmax(gam, 0.0)));
            double gam_prev = 1.0, alpha_prev = 1.0;
            int k = 0;
            bool broke = false;
            while (sqrt(fmax(gam, 0.0)) > thr && k < P.cg_max) {
                double dl[1];
                const int op1[1] = {0};
                if (cbcg) {
                    // column-blocked passes: u'Mu = ||A_hat'u||^2 is known after
                    // the first half, the second half's sums are combined in the
                    // vector step
                    phase_cg_At_cb(P);                          // partial sums of A'u
                    ++nAT;
                    ACS_SYNC(PH_CG_AT);
                    phase_cg_tcomb(P);                          // t = O^2 A'u, u'Mu
                    ACS_SYNC(PH_CG_TCOMB);
                    grid_combine<1>(P.partials, op1, dl);
                } else {
                    phase_cg_At(P);                             // t = O^2 A' u
                    ++nAT;
                    ACS_SYNC(PH_CG_AT);
                    phase_cg_A(P);                              // au = A t = M u
                    ++nA;
                    ACS_SYNC(PH_CG_A);
                    grid_combine<1>(P.partials, op1, dl);
                }
                const double beta = (k == 0) ? 0.0 : gam / gam_prev;
                const double denom = dl[0] - ((k == 0) ? 0.0 : beta * gam / alpha_prev);
                if (!(denom > 0.0)) {
                    // p'Mp <= 0 in finite precision: the solve has reached its
                    // attainable accuracy (or M is singular along p); keep w --
                    // the next FP64 residual carries on from it
                    broke = true;
                    break;
                }
                const double alpha = gam / denom;
                if (cbcg) {
                    phase_cg_A_cb(P);                           // partial sums of A t = M u
                    ++nA;
                    ACS_SYNC(PH_CG_A);
                    phase_cg_vec<T, true>(P, alpha, (T)beta);
                } else {
                    phase_cg_vec<T, false>(P, alpha, (T)beta);
                }
                ACS_SYNC(PH_CG_VEC);
                double gn[1];
                grid_combine<1>(P.partials, op1, gn);
                gam_prev = gam;
                alpha_prev = alpha;
                gam = gn[0];
                ++k;
                if (!isfinite(gam)) { status = ACS_ERR_NUMERICAL; break; }
            }
            if (!ok || status == ACS_ERR_NUMERICAL) break;
            cg_total += k;
            win_cg += k;
            // an FP32 solve that stalls far above its target cannot refine this M
            if ((broke || k >= P.cg_max) && sqrt(fmax(gam, 0.0)) > 100.0 * thr) trouble = true;
        }
        if (!ok || status == ACS_ERR_NUMERICAL) break;

        const bool check = (lnext % P.check_every == 0) || (lnext == P.max_iter);
        const bool want_xz = check || in_schedule(P, lnext + 1);
        // step 17 of the next iteration in this pass's epilogue (orthant-only,
        // no extrapolation, no rescaling at the next iteration)
        const bool fuse_abs = P.n_soc == 0 && !P.admm && P.extrap == 0.0 && !in_schedule(P, lnext + 1);
        if (outer32) {                                          // steps 18-21, FP32 product
            phase_update_cb(P);
            ++nAT32;
            ACS_SYNC(PH_UPDATE);
            phase_update_comb(P, want_xz, fuse_abs);
            ACS_SYNC(PH_UPD_COMB);
        } else if (outer32_l2) {
            phase_update_f32(P, want_xz, fuse_abs);             // steps 18-21, FP32 product
            ++nAT32;
            ACS_SYNC(PH_UPDATE);
        } else {
            phase_update(P, true, want_xz, fuse_abs);          // steps 18-21
            ++nAT64;
            ACS_SYNC(PH_UPDATE);
        }
        abs_fused = fuse_abs;
        {
            double d2[3];
            const int op[3] = {0, 0, 1};
            grid_combine<3>(P.partials, op, d2);
            if (P.admm && P.n_soc > 0) {                        // the cones' share of the update
                phase_admm_soc(P, want_xz);
                ACS_SYNC(PH_UPDATE);
                double e2[2];
                const int op2[2] = {0, 0};
                grid_combine<2>(P.partials, op2, e2);
                d2[0] += e2[0];
                d2[1] += e2[1];
            }
            const double ds_new = sqrt(d2[0]);
            snorm = sqrt(d2[1]);
            over = d2[2] > 0.0;
            if (!isfinite(ds_new) || !isfinite(snorm)) { status = ACS_ERR_NUMERICAL; l = lnext; break; }
            // With exact projections the step norm ||s_l - s_{l-1}|| never grows
            // between rescalings (the iteration map is firmly nonexpansive,
            // Lemma 3); growth beyond what the allowed error explains means the
            // CG error estimate (J-norm of the residual) is too optimistic for
            // this M, so the rule is tightened for the rest of the solve.
            // In the FP32 solve a factor below 1e-4 * cg_eta means the FP32
            // correction cannot reach the accuracy this M needs: the solve
            // continues with an FP64 correction solve instead.
            if (!cond && isfinite(ds) && ds_new > (1.0 + 4.0 * eta) * ds && eta > 1e-8) {
                if (sizeof(T) == 4 && eta <= 1e-4 * P.cg_eta * 1.0000001) trouble = true;
                else eta *= 0.1;
            }
            ds = ds_new;
        }
        l = lnext;
        ++win_it;
        if (sizeof(T) == 4 && trouble && P.switch_ok) { status = ST_SWITCH; break; }

        if (check) {
            phase_kkt(P);
            ++nA64;
            ++nAT64;
            ++nchk;
            ACS_SYNC(PH_KKT);
            double r8[8];
            const int op[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            grid_combine<8>(P.partials, op, r8);
            res[0] = sqrt(r8[0]) / (1.0 + P.bnorm);
            res[1] = sqrt(r8[1]) / (1.0 + P.cnorm);
            res[2] = fabs(r8[2] - r8[3]) / (1.0 + fabs(r8[2]) + fabs(r8[3]));
            res[3] = fmax(sqrt(r8[4]), sqrt(r8[5])) / (1.0 + fmax(sqrt(r8[6]), sqrt(r8[7])));
            res[4] = r8[2];
            res[5] = r8[3];
            const double mx = fmax(fmax(res[0], res[1]), fmax(res[2], res[3]));
            if (!isfinite(mx)) { status = ACS_ERR_NUMERICAL; break; }
            if (mx <= P.tol) { status = ACS_SOLVED; break; }
            // FP32 outer passes end once the residuals reach outer32_tol, or
            // once they stop falling (the FP32 products' rounding floor): the
            // rest of the solve runs the FP64 passes from the same iterate
            if (outer32) {
                if (mx < 0.9 * best_mx) {
                    best_mx = mx;
                    flat_checks = 0;
                } else {
                    ++flat_checks;
                }
                if (mx <= P.outer32_tol || flat_checks >= kOuter32FlatChecks) {
                    outer32 = false;
                    outer32_end = l;
                }
            }
        }
        if (over && l < P.max_iter) { status = ST_PAUSED; break; }
    }
#undef ACS_SYNC

    if (clock_owner) {
        const int err = ld_volatile_int(&ctl->err);
        ctl->status = err != 0 ? err : status;
        if (status == ST_SWITCH && err == 0) ctl->switched_at = l;
        ctl->l = l;
        ctl->cg_iters += cg_total;
        for (int i = 0; i < 6; ++i) ctl->res[i] = res[i];
        ctl->ds = ds;
        ctl->snorm = snorm;
        ctl->eta = eta;
        ctl->n_cg_A += nA;
        ctl->n_cg_AT += nAT;
        ctl->n_64_A += nA64;
        ctl->n_64_AT += nAT64;
        ctl->n_cond += ncond;
        ctl->n_checks += nchk;
        ctl->n_dense_solve += ndense;
        ctl->n_dense_factor += nfactor;
        ctl->n_32_A += nA32;
        ctl->n_32_AT += nAT32;
        ctl->outer32_end = outer32_end;
        ctl->stage = (sizeof(T) == 8 || status == ST_SWITCH) ? 1 : 0;
        ctl->dense_on = (dense || want_dense) ? 1 : 0;
        ctl->factor_ok = factor_ok ? 1 : 0;
        ctl->dense_failed = dense_failed ? 1 : 0;
        ctl->win_cg = win_cg;
        ctl->win_it = win_it;
        ctl->extrap_ok = extrap_ok ? 1 : 0;
        ctl->bar_gen = sync_smem().gen;
        for (int i = 0; i < PH_COUNT; ++i) {
            ctl->phase_ns[i] += s_ph_ns[i];
            ctl->phase_n[i] += s_ph_n[i];
        }
    }
    return status;
}

}  // namespace acs
