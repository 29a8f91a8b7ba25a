// Launches in which fixed teams of CTAs solve many independent programs:
// the device side (team kernel, reset kernels, the initial point) and the
// host-side member layout shared by the batched API (acs_batch.cu) and the
// serving loop (acs_serve.cu).  Everything has internal linkage: each of the
// two translation units holds its own copy.  Not part of the public ABI.
#pragma once

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "acs_device.cuh"
#include "acs_host.cuh"

namespace acs {
namespace {

// ---------------------------------------------------------------------------
// device
// ---------------------------------------------------------------------------

struct BatchArgs {
    int count;                        // members
    const int* order;                 // [count] members in the order teams take them
    const IterParams<float>* p32;     // [count] parameters of the FP32-correction loop
    const IterParams<double>* p64;    // [count] parameters of the FP64-correction loop
    Control* ctl;                     // [count]
    int* head;                        // next position in order
    int* mailbox;                     // [teams] member posted by the team's rank 0
    unsigned long long* team_bar;     // [teams] barrier arrival counters
    double* team_part;                // [CTAs * kMaxRed] partials
    int* team_err;                    // [teams] barrier failures outside a member's solve
    double* dense;                    // [teams * 2 * dense_m2] scratch of the cached operator
    long long dense_m2;               // (largest m among members that use it)^2
    unsigned long long* round_t0;     // time-sliced launch: global-timer start of the launch
    unsigned long long round_ns;      //   and its length (0 = run every member to its end)
    const int* cta_k;                 // assigned teams: per CTA, position in order (-1 = idle),
    const int* cta_rank;              //   rank in its team,
    const int* cta_g;                 //   and team size; NULL = queued teams of g CTAs
    int g;                            // CTAs per team
    int fp64;                         // FP64 correction solve from the start
};

__global__ void batch_reset(BatchArgs B, double eta0) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = t; i < B.count; i += gridDim.x * blockDim.x) {
        Control* c = B.ctl + i;
        c->status = ST_RUNNING;
        c->err = 0;
        c->l = 0;
        c->cg_iters = 0;
        c->switched_at = 0;
        for (int k = 0; k < 6; ++k) c->res[k] = NAN;
        c->ds = INFINITY;
        c->snorm = 0.0;
        c->eta = eta0;
        c->n_cg_A = c->n_cg_AT = c->n_64_A = c->n_64_AT = c->n_cond = c->n_checks = 0;
        for (int k = 0; k < PH_COUNT; ++k) { c->phase_ns[k] = 0; c->phase_n[k] = 0; }
        c->bar_count = 0;
        c->bar_gen = 0;
        c->bar_count64 = 0;
        c->stage = 0;
        c->dense_on = 0;
        c->dense_failed = 0;
        c->win_it = 0;
        c->win_cg = 0;
        c->extrap_ok = 0;
        c->factor_ok = 0;
    }
    if (t == 0) *B.head = 0;
}

__global__ void batch_reset_teams(BatchArgs B, int teams) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < teams; t += gridDim.x * blockDim.x) {
        B.team_bar[t] = 0ull;
        B.team_err[t] = 0;
        B.mailbox[t] = 0;
    }
}

// Initial point of Algorithm 2 (x = z = e, the cone identity; w = q = 0),
// written by the whole team.
template <typename T>
__device__ void init_member(const IterParams<T>& P) {
    for (int j = global_tid(); j < P.n_orth; j += global_threads()) {
        P.x[j] = 1.0;
        P.z[j] = 1.0;
        P.X.q[j] = 0.0;
    }
    const int lane = threadIdx.x & 31;
    for (int cI = global_warp(); cI < P.n_soc; cI += global_warps()) {
        const int a = __ldg(P.soc_off + cI), e = __ldg(P.soc_off + cI + 1);
        for (int j = a + lane; j < e; j += 32) {
            const double v = (j == a) ? 1.0 : 0.0;
            P.x[j] = v;
            P.z[j] = v;
            P.X.q[j] = 0.0;
        }
    }
    for (int i = global_tid(); i < P.m; i += global_threads()) P.X.w[i] = 0.0;
}

// One member's solve (or its time slice) by the calling team.  Returns false
// if the team must stop (a barrier failed or timed out).
__device__ __noinline__ bool run_member(const BatchArgs& B, int i, double* scratch, unsigned long long deadline) {
    Control* ctl = B.ctl + i;
    sync_init(sync_smem().gen);                          // clear a failure of the previous member
    if (threadIdx.x == 0) {
        SyncShared& S = sync_smem();
        // a member with scratch of its own keeps its cached factor across launches
        S.dM = B.p64[i].dM ? B.p64[i].dM : scratch;
        S.dX = B.p64[i].dX ? B.p64[i].dX : (scratch ? scratch + B.dense_m2 : nullptr);
        S.deadline = deadline;
    }
    __syncthreads();
    // a resumed member (refresh) continues in the loop it paused in
    const bool fresh = B.p64[i].refresh == 0;
    const int stage = fresh ? 0 : __ldcg(&ctl->stage);
    if (B.fp64 || B.p64[i].dense == 1 || stage == 1) {   // the cached operator runs in the FP64 loop
        const IterParams<double>& P = B.p64[i];
        if (fresh) init_member(P);
        if (!grid_sync(&ctl->err)) return false;
        solve_loop<double>(P, ST_RUNNING);
    } else {
        const IterParams<float>& P = B.p32[i];
        if (fresh) init_member(P);
        if (!grid_sync(&ctl->err)) return false;
        if (solve_loop<float>(P, ST_RUNNING) == ST_SWITCH) {
            // the loop's state is in ctl (written by rank 0): publish it
            if (!grid_sync(&ctl->err)) return false;
            solve_loop<double>(B.p64[i], ST_SWITCH);
        }
    }
    // a barrier that timed out leaves the team out of step: stop it
    return ld_volatile_int(&ctl->err) != ACS_ERR_DEVICE_TIMEOUT;
}

__device__ __forceinline__ unsigned long long launch_deadline(const BatchArgs& B) {
    __shared__ unsigned long long s_deadline;
    if (threadIdx.x == 0) {
        s_deadline = 0ull;
        if (B.round_ns) {
            // the first CTA to start fixes the launch's start time
            const unsigned long long now = gtimer();
            const unsigned long long t0 = atomicCAS(B.round_t0, 0ull, now);
            s_deadline = (t0 == 0ull ? now : t0) + B.round_ns;
        }
    }
    __syncthreads();
    return s_deadline;
}

// Two ways to map CTAs to members.  Queued teams (cta_k == NULL): fixed teams
// of g consecutive CTAs take members from a global counter until none is
// left (or the time slice is over).  Assigned teams (cta_k != NULL): the host
// has given every member a team of its own, cta_g[b] consecutive CTAs sized
// by its work (a launch with fewer members than CTAs), and CTA b works as
// rank cta_rank[b] on member order[cta_k[b]] (or idles if cta_k[b] < 0).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) batch_kernel(BatchArgs B) {
    if (B.cta_k) {
        const int k = __ldg(B.cta_k + blockIdx.x);
        if (k < 0) return;
        const int rank = __ldg(B.cta_rank + blockIdx.x), g = __ldg(B.cta_g + blockIdx.x);
        const int base = (int)blockIdx.x - rank;
        team_set(rank, g, B.team_bar + base, B.team_part + (size_t)base * kMaxRed, nullptr, nullptr);
        sync_init(0u);
        const unsigned long long deadline = launch_deadline(B);
        run_member(B, __ldg(B.order + k), nullptr, deadline);
        return;
    }
    const int team = (int)blockIdx.x / B.g, rank = (int)blockIdx.x % B.g;
    double* scratch = B.dense ? B.dense + (size_t)team * 2 * B.dense_m2 : nullptr;
    team_set(rank, B.g, B.team_bar + team, B.team_part + (size_t)team * B.g * kMaxRed, scratch,
             scratch ? scratch + B.dense_m2 : nullptr);
    sync_init(0u);
    __shared__ int s_k;
    const unsigned long long deadline = launch_deadline(B);
    while (true) {
        // the team's rank 0 takes the next member (none once the time slice
        // is over); the barrier publishes it
        if (rank == 0 && threadIdx.x == 0)
            B.mailbox[team] = (deadline && gtimer() > deadline) ? B.count : atomicAdd(B.head, 1);
        if (!grid_sync(B.team_err + team)) return;
        if (threadIdx.x == 0) s_k = __ldcg(B.mailbox + team);
        __syncthreads();
        const int k = s_k;
        if (k >= B.count) return;
        if (!run_member(B, __ldg(B.order + k), scratch, deadline)) return;
    }
}

// ---------------------------------------------------------------------------
// host-side member layout
// ---------------------------------------------------------------------------

constexpr int kThreadChoices[3] = {256, 512, 1024};
constexpr int kTeamChoices[3] = {1, 2, 4};

// Bump allocator over one device allocation; a dry run (base = 0) measures.
struct Pool {
    char* base = nullptr;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base + off);
        off += (count ? count : 1) * sizeof(T);
        return p;
    }
};

struct DevSell {      // offsets of one sliced-ELLPACK matrix inside the pool
    int* sptr; int* slen; int* col; float* v32; double* v64; unsigned short* v16;
};

// Device layout of one matrix: FP64 values, and FP32 values or BF16 bits.
inline void layout_sell(Pool& P, const host::HostSell& H, DevSell& D, bool bf16) {
    D.sptr = P.take<int>(H.sptr.size());
    D.slen = P.take<int>(H.slen.size());
    D.col = P.take<int>(H.col.size());
    D.v32 = bf16 ? nullptr : P.take<float>(H.col.size());
    D.v16 = bf16 ? P.take<unsigned short>(H.col.size()) : nullptr;
    D.v64 = P.take<double>(H.col.size());
}

template <typename T>
void put_bytes(char* img, const void* dev_off, const T* src, size_t count);

// Host image of one matrix at the offsets of layout_sell.
template <typename Img>
void image_sell(Img& img, const host::HostSell& H, const DevSell& D) {
    put_bytes(img.data(), D.sptr, H.sptr.data(), H.sptr.size());
    put_bytes(img.data(), D.slen, H.slen.data(), H.slen.size());
    put_bytes(img.data(), D.col, H.col.data(), H.col.size());
    if (D.v16) {
        std::vector<unsigned short> h(H.val.size());
        for (size_t k = 0; k < h.size(); ++k) h[k] = host::to_bf16(H.val[k]);
        put_bytes(img.data(), D.v16, h.data(), h.size());
    } else {
        std::vector<float> f(H.val.size());
        for (size_t k = 0; k < f.size(); ++k) f[k] = (float)H.val[k];
        put_bytes(img.data(), D.v32, f.data(), f.size());
    }
    put_bytes(img.data(), D.v64, H.val.data(), H.val.size());
}

// Device addresses of a matrix laid out at offsets from base.
template <typename T>
T* rebase(T* off, char* base);
inline void rebase_sell(const DevSell& D, char* base, SellMat& S) {
    S.sptr = rebase(D.sptr, base); S.slen = rebase(D.slen, base); S.col = rebase(D.col, base);
    S.v32 = D.v32 ? rebase(D.v32, base) : nullptr;
    S.v16 = D.v16 ? rebase(D.v16, base) : nullptr;
    S.v64 = rebase(D.v64, base);
}

struct Matrix {       // one distinct A of the batch
    host::HostProblem H;            // host image (released after upload)
    SellMat A{}, AT{};
    DevSell dA{}, dAT{};
    long long stored = 0;
};

struct Member {
    int m = 0, n = 0, n_orth = 0, n_soc = 0, mat = 0;
    int dense = 0;                    // cached dense operator: 0 never, 1 always, 2 when CG stalls
    long long nnz = 0;
    std::vector<double> b, c;
    std::vector<int> soc_off;
    double bnorm = 0, cnorm = 0;
    // device pointers inside the pool
    double *db = nullptr, *dc = nullptr, *x = nullptr, *z = nullptr, *ocone = nullptr;
    int* dsoc = nullptr;
    Outer X{};
    Inner<float> V32{};
    Inner<double> V64{};
};

int occupancy_for(int threads, int* blocks_per_sm) {
    cudaError_t e = cudaErrorInvalidValue;
    if (threads == 256) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel<256>, 256, 0);
    if (threads == 512) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel<512>, 512, 0);
    if (threads == 1024) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel<1024>, 1024, 0);
    return e == cudaSuccess && *blocks_per_sm >= 1 ? ACS_SOLVED : ACS_ERR_CUDA;
}

const void* kernel_for(int threads) {
    if (threads == 256) return (const void*)batch_kernel<256>;
    if (threads == 512) return (const void*)batch_kernel<512>;
    return (const void*)batch_kernel<1024>;
}

// Final status of a member from its control block (a solve that never ended
// -- running, handed over, or paused at a deadline -- is reported as an error
// by the batched API; the serving loop resumes paused ones instead).
int member_status(const Control& C) {
    int s = C.status;
    if (s == ST_RUNNING || s == ST_SWITCH || s == ST_PAUSED) s = ACS_ERR_CUDA;
    return s;
}

bool valid_mapping(const acs_batch_mapping& m) {
    const bool t = m.threads_per_cta == 256 || m.threads_per_cta == 512 || m.threads_per_cta == 1024;
    const bool g = m.team_ctas == 1 || m.team_ctas == 2 || m.team_ctas == 4 || m.team_ctas == 8;
    return t && g;
}

template <typename T>
IterParams<T> member_params(const acs_settings& set, const int* d_cond_list, int n_cond_list, const Member& M,
                            const Matrix& X, const Inner<T>& V, double tol, int max_iter) {
    IterParams<T> Q{};
    Q.m = M.m; Q.n = M.n; Q.n_orth = M.n_orth; Q.n_soc = M.n_soc;
    Q.A = X.A; Q.AT = X.AT;
    Q.soc_off = M.dsoc;
    Q.b = M.db; Q.c = M.dc; Q.bnorm = M.bnorm; Q.cnorm = M.cnorm;
    Q.X = M.X;
    Q.V = V;
    Q.x = M.x; Q.z = M.z; Q.ocone = M.ocone;
    Q.partials = nullptr; Q.flags = nullptr; Q.release = nullptr; Q.bcast = nullptr;
    Q.ctl = nullptr;
    Q.mu = set.mu; Q.t_cond = set.t;
    Q.cond_first = set.cond_first; Q.cond_period = set.cond_period;
    Q.cond_list = d_cond_list; Q.n_cond_list = n_cond_list;
    Q.check_every = set.check_every > 0 ? set.check_every : 1;
    Q.max_iter = max_iter;
    Q.tol = tol;
    Q.cg_eta = set.cg_eta;
    Q.cg_tol = set.cg_tol;
    Q.cg_relfloor = sizeof(T) == 4 ? 1e-6 : 1e-13;
    Q.cg_max = set.cg_max_iter;
    Q.refresh = 0;
    Q.refine = set.cg_refine > 0 ? set.cg_refine : 1;
    Q.switch_ok = set.precision != ACS_PREC_FP64 ? 1 : 0;
    Q.dense = M.dense;
    Q.switch_budget = host::switch_budget(set, M.m, M.nnz);
    Q.extrap = set.extrapolation;
    Q.admm = set.splitting == ACS_SPLIT_ADMM ? 1 : 0;
    Q.dM = Q.dX = nullptr;                    // team scratch, set by the kernel
    return Q;
}

template <typename T>
void put_bytes(char* img, const void* dev_off, const T* src, size_t count) {
    if (count) memcpy(img + reinterpret_cast<size_t>(dev_off), src, count * sizeof(T));
}

template <typename T>
T* rebase(T* off, char* base) {
    return reinterpret_cast<T*>(base + reinterpret_cast<size_t>(off));
}

}  // namespace
}  // namespace acs
