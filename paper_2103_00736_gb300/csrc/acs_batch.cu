// Batched solves: many independent conic programs of uneven sizes in one
// persistent launch, replayed from a captured CUDA graph.
//
// Device design.  The launch is one cooperative grid of resident CTAs split
// into fixed teams of g consecutive CTAs (g = 1 for most batches).  A team's
// rank-0 CTA takes the next member from a global counter (members ordered by
// decreasing size, so the longest solves start first and the tail is short),
// posts it to the team, and the team runs that member's whole solve --
// Algorithm 2 (arXiv 2103.00736, Section IV) with the same phases as the
// single-problem kernel -- synchronising only among its own CTAs (a team of
// one CTA needs no global barrier at all).  Then it takes the next member.
// The mixed-precision hand-over (FP32 correction solve -> FP64) happens inside
// the same launch.  Members sharing one A point at a single device copy of it,
// so their matrix passes hit in L2.
//
// Host design.  Every member is prepared like a single problem (validation,
// relabelled rows, sliced-ELLPACK A and A'), then all device data live in one
// allocation: a static region (matrices, b, c, cone offsets) uploaded once
// from a host image, and a state region (iterates, solver vectors) zeroed once.

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <numeric>
#include <type_traits>
#include <vector>

#include "acs_device.cuh"
#include "acs_host.cuh"

namespace acs {

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

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) batch_kernel(BatchArgs B) {
    const int team = (int)blockIdx.x / B.g, rank = (int)blockIdx.x % B.g;
    double* scratch = B.dense ? B.dense + (size_t)team * 2 * B.dense_m2 : nullptr;
    team_set(rank, B.g, B.team_bar + team, B.team_part + (size_t)team * B.g * kMaxRed, scratch,
             scratch ? scratch + B.dense_m2 : nullptr);
    sync_init(0u);
    __shared__ int s_k;
    while (true) {
        // the team's rank 0 takes the next member; the barrier publishes it
        if (rank == 0 && threadIdx.x == 0) B.mailbox[team] = atomicAdd(B.head, 1);
        if (!grid_sync(B.team_err + team)) return;
        if (threadIdx.x == 0) s_k = __ldcg(B.mailbox + team);
        __syncthreads();
        const int k = s_k;
        if (k >= B.count) return;
        const int i = __ldg(B.order + k);
        Control* ctl = B.ctl + i;
        sync_init(sync_smem().gen);                      // clear a failure of the previous member
        int st;
        if (B.fp64 || B.p64[i].dense == 1) {             // the cached operator runs in the FP64 loop
            const IterParams<double>& P = B.p64[i];
            init_member(P);
            if (!grid_sync(&ctl->err)) return;
            st = solve_loop<double>(P, ST_RUNNING);
        } else {
            const IterParams<float>& P = B.p32[i];
            init_member(P);
            if (!grid_sync(&ctl->err)) return;
            st = solve_loop<float>(P, ST_RUNNING);
            if (st == ST_SWITCH) {
                // the loop's state is in ctl (written by rank 0): publish it
                if (!grid_sync(&ctl->err)) return;
                solve_loop<double>(B.p64[i], ST_SWITCH);
            }
        }
        // a barrier that timed out leaves the team out of step: stop it
        if (ld_volatile_int(&ctl->err) == ACS_ERR_DEVICE_TIMEOUT) return;
    }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------

namespace {

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
    int* sptr; int* slen; int* col; float* v32; double* v64;
};

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

}  // namespace

struct Batch {
    int count = 0, device = 0, nsm = 0;
    acs_settings set{};
    std::vector<int> cond_list_host;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<Matrix> mats;
    std::vector<Member> mem;
    std::vector<int> order;
    // pool
    char* pool = nullptr;
    size_t static_bytes = 0, total_bytes = 0;
    int* d_cond_list = nullptr;
    int* d_order = nullptr;
    IterParams<float>* d_p32 = nullptr;
    IterParams<double>* d_p64 = nullptr;
    Control* d_ctl = nullptr;
    int* d_head = nullptr;
    int* d_mailbox = nullptr;
    unsigned long long* d_team_bar = nullptr;
    double* d_team_part = nullptr;
    int* d_team_err = nullptr;
    double* d_dense = nullptr;
    long long dense_m2 = 0;
    int max_ctas = 0;
    // mapping and launch
    acs_batch_mapping map{1024, 1};
    int grid = 0;
    double p_tol = -1.0;
    int p_max_iter = -1;
    cudaGraphExec_t gexec = nullptr;
    bool graph_ok = false, last_graph = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    std::vector<Control> ctl_host;
};

namespace {

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

bool valid_mapping(const acs_batch_mapping& m) {
    const bool t = m.threads_per_cta == 256 || m.threads_per_cta == 512 || m.threads_per_cta == 1024;
    const bool g = m.team_ctas == 1 || m.team_ctas == 2 || m.team_ctas == 4 || m.team_ctas == 8;
    return t && g;
}

// CTAs of a launch under mapping m: every resident CTA, in whole teams.
int grid_for(Batch* B, const acs_batch_mapping& m, int* grid) {
    int bps = 0;
    if (occupancy_for(m.threads_per_cta, &bps) != ACS_SOLVED) return ACS_ERR_CUDA;
    int g = B->nsm * bps;
    g -= g % m.team_ctas;
    if (g < m.team_ctas || g > B->max_ctas) return ACS_ERR_ARG;
    *grid = g;
    return ACS_SOLVED;
}

template <typename T>
IterParams<T> member_params(const Batch* B, const Member& M, const Matrix& X, const Inner<T>& V, double tol,
                            int max_iter) {
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
    Q.mu = B->set.mu; Q.t_cond = B->set.t;
    Q.cond_first = B->set.cond_first; Q.cond_period = B->set.cond_period;
    Q.cond_list = B->d_cond_list; Q.n_cond_list = (int)B->cond_list_host.size();
    Q.check_every = B->set.check_every > 0 ? B->set.check_every : 1;
    Q.max_iter = max_iter;
    Q.tol = tol;
    Q.cg_eta = B->set.cg_eta;
    Q.cg_tol = B->set.cg_tol;
    Q.cg_relfloor = sizeof(T) == 4 ? 1e-6 : 1e-13;
    Q.cg_max = B->set.cg_max_iter;
    Q.refresh = 0;
    Q.refine = B->set.cg_refine > 0 ? B->set.cg_refine : 1;
    Q.switch_ok = B->set.precision == ACS_PREC_MIXED ? 1 : 0;
    Q.dense = M.dense;
    Q.dense_switch_cg = B->set.dense_switch_cg;
    Q.dM = Q.dX = nullptr;                    // team scratch, set by the kernel
    return Q;
}

// Write the per-member parameter blocks for (tol, max_iter).
int upload_params(Batch* B, double tol, int max_iter) {
    std::vector<IterParams<float>> p32(B->count);
    std::vector<IterParams<double>> p64(B->count);
    for (int i = 0; i < B->count; ++i) {
        const Member& M = B->mem[i];
        p32[i] = member_params<float>(B, M, B->mats[M.mat], M.V32, tol, max_iter);
        p64[i] = member_params<double>(B, M, B->mats[M.mat], M.V64, tol, max_iter);
        p32[i].ctl = B->d_ctl + i;
        p64[i].ctl = B->d_ctl + i;
    }
    if (cudaMemcpyAsync(B->d_p32, p32.data(), sizeof(p32[0]) * B->count, cudaMemcpyHostToDevice, B->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(B->d_p64, p64.data(), sizeof(p64[0]) * B->count, cudaMemcpyHostToDevice, B->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(B->stream) != cudaSuccess)
        return ACS_ERR_CUDA;
    B->p_tol = tol;
    B->p_max_iter = max_iter;
    return ACS_SOLVED;
}

BatchArgs batch_args(Batch* B) {
    BatchArgs a{};
    a.count = B->count;
    a.order = B->d_order;
    a.p32 = B->d_p32;
    a.p64 = B->d_p64;
    a.ctl = B->d_ctl;
    a.head = B->d_head;
    a.mailbox = B->d_mailbox;
    a.team_bar = B->d_team_bar;
    a.team_part = B->d_team_part;
    a.team_err = B->d_team_err;
    a.dense = B->dense_m2 > 0 ? B->d_dense : nullptr;
    a.dense_m2 = B->dense_m2;
    a.g = B->map.team_ctas;
    a.fp64 = B->set.precision == ACS_PREC_FP64 ? 1 : 0;
    return a;
}

// Reset + persistent launch on the batch's stream (captured or direct).
cudaError_t enqueue(Batch* B) {
    BatchArgs a = batch_args(B);
    const int teams = B->grid / B->map.team_ctas;
    batch_reset<<<(B->count + 255) / 256, 256, 0, B->stream>>>(a, B->set.cg_eta);
    batch_reset_teams<<<(teams + 255) / 256, 256, 0, B->stream>>>(a, teams);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a};
    return cudaLaunchCooperativeKernel(kernel_for(B->map.threads_per_cta), dim3(B->grid),
                                       dim3(B->map.threads_per_cta), args, 0, B->stream);
}

void drop_graph(Batch* B) {
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    B->gexec = nullptr;
    B->graph_ok = false;
}

int set_mapping(Batch* B, const acs_batch_mapping& m) {
    if (!valid_mapping(m)) return ACS_ERR_ARG;
    int grid = 0;
    const int rc = grid_for(B, m, &grid);
    if (rc != ACS_SOLVED) return rc;
    if (m.threads_per_cta != B->map.threads_per_cta || m.team_ctas != B->map.team_ctas) drop_graph(B);
    B->map = m;
    B->grid = grid;
    return ACS_SOLVED;
}

int launch(Batch* B, double tol, int max_iter, bool use_graph) {
    if (tol != B->p_tol || max_iter != B->p_max_iter) {
        drop_graph(B);
        const int rc = upload_params(B, tol, max_iter);
        if (rc != ACS_SOLVED) return rc;
    }
    cudaStream_t st = B->stream;
    if (use_graph && !B->gexec) {
        // capture once; if capturing the cooperative launch is refused, the
        // work is launched directly instead (reported by acs_batch_info)
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const cudaError_t e1 = enqueue(B);
            const cudaError_t e2 = cudaStreamEndCapture(st, &g);
            if (e1 == cudaSuccess && e2 == cudaSuccess && g &&
                cudaGraphInstantiate(&B->gexec, g, 0) == cudaSuccess) {
                B->graph_ok = true;
            } else {
                B->gexec = nullptr;
            }
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
    }
    cudaEventRecord(B->ev[0], st);
    cudaError_t e;
    if (use_graph && B->gexec) {
        e = cudaGraphLaunch(B->gexec, st);
        B->last_graph = true;
    } else {
        e = enqueue(B);
        B->last_graph = false;
    }
    cudaEventRecord(B->ev[1], st);
    if (e != cudaSuccess) {
        fprintf(stderr, "acs: batched launch failed: %s\n", cudaGetErrorString(e));
        return ACS_ERR_CUDA;
    }
    return ACS_SOLVED;
}

int fetch_controls(Batch* B) {
    B->ctl_host.resize(B->count);
    if (cudaMemcpyAsync(B->ctl_host.data(), B->d_ctl, sizeof(Control) * B->count, cudaMemcpyDeviceToHost,
                        B->stream) != cudaSuccess ||
        cudaStreamSynchronize(B->stream) != cudaSuccess)
        return ACS_ERR_CUDA;
    return ACS_SOLVED;
}

int member_status(const Control& C) {
    int s = C.status;
    if (s == ST_RUNNING || s == ST_SWITCH) s = ACS_ERR_CUDA;   // never finished
    return s;
}

// Lay out (dry run with base = 0, then for real) every device buffer.
void layout(Batch* B, Pool& P) {
    const int count = B->count;
    // static region: matrices, then per-member b, c, cone offsets, cond list
    for (Matrix& X : B->mats) {
        auto put = [&](const host::HostSell& H, DevSell& D) {
            D.sptr = P.take<int>(H.sptr.size());
            D.slen = P.take<int>(H.slen.size());
            D.col = P.take<int>(H.col.size());
            D.v32 = P.take<float>(H.col.size());
            D.v64 = P.take<double>(H.col.size());
        };
        put(X.H.A, X.dA);
        put(X.H.AT, X.dAT);
    }
    for (Member& M : B->mem) {
        M.db = P.take<double>(M.m);
        M.dc = P.take<double>(M.n);
        M.dsoc = P.take<int>(M.n_soc + 1);
    }
    B->d_cond_list = P.take<int>(B->cond_list_host.size());
    B->d_order = P.take<int>(count);
    B->static_bytes = P.off;
    // state region
    for (Member& M : B->mem) {
        const int m = M.m, n = M.n;
        M.x = P.take<double>(n);
        M.z = P.take<double>(n);
        M.ocone = P.take<double>((size_t)M.n_orth + M.n_soc);
        Outer& X = M.X;
        X.s = P.take<double>(n); X.p = P.take<double>(n); X.g = P.take<double>(n);
        X.q = P.take<double>(n); X.chat = P.take<double>(n); X.O = P.take<double>(n);
        X.w = P.take<double>(m); X.btil = P.take<double>(m);
        auto inner = [&](auto& V) {
            using T = std::remove_pointer_t<decltype(V.r)>;
            V.r = P.take<T>(m); V.u = P.take<T>(m); V.p = P.take<T>(m); V.sv = P.take<T>(m);
            V.au = P.take<T>(m); V.jinv = P.take<T>(m); V.t = P.take<T>(n); V.O2 = P.take<T>(n);
        };
        inner(M.V32);
        inner(M.V64);
    }
    B->d_p32 = P.take<IterParams<float>>(count);
    B->d_p64 = P.take<IterParams<double>>(count);
    B->d_ctl = P.take<Control>(count);
    B->d_head = P.take<int>(32);
    B->d_mailbox = P.take<int>(B->max_ctas);
    B->d_team_bar = P.take<unsigned long long>(B->max_ctas);
    B->d_team_part = P.take<double>((size_t)B->max_ctas * kMaxRed);
    B->d_team_err = P.take<int>(B->max_ctas);
    B->d_dense = P.take<double>(B->dense_m2 > 0 ? (size_t)B->max_ctas * 2 * B->dense_m2 : 1);
    B->total_bytes = P.off;
}

template <typename T>
void put_bytes(std::vector<char>& img, const void* dev_off, const T* src, size_t count) {
    if (count) memcpy(img.data() + reinterpret_cast<size_t>(dev_off), src, count * sizeof(T));
}

void free_batch(Batch* B) {
    if (!B) return;
    drop_graph(B);
    if (B->pool) cudaFree(B->pool);
    B->pool = nullptr;
    for (auto& e : B->ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
    B->stream = nullptr;
}

template <typename T>
T* rebase(T* off, char* base) {
    return reinterpret_cast<T*>(base + reinterpret_cast<size_t>(off));
}

}  // namespace
}  // namespace acs

using acs::Batch;

extern "C" {

int acs_batch_create(int32_t count, const acs_instance* members, const acs_settings* settings,
                     const acs_batch_mapping* mapping, acs_batch** out, int32_t* bad_member) {
    using namespace acs;
    if (bad_member) *bad_member = -1;
    if (!out) return ACS_ERR_ARG;
    *out = nullptr;
    if (count <= 0 || !members) return ACS_ERR_ARG;
    acs_settings set;
    if (settings) set = *settings; else acs_settings_default(&set);
    if (!host::valid_settings(set)) return ACS_ERR_ARG;
    acs_batch_mapping map0 = mapping ? *mapping : acs_batch_mapping{1024, 1};
    if (!valid_mapping(map0)) return ACS_ERR_ARG;

    Batch* B = new (std::nothrow) Batch();
    if (!B) return ACS_ERR_OOM;
    B->count = count;
    B->set = set;
    B->device = set.device;
    if (set.n_cond_list > 0) B->cond_list_host.assign(set.cond_list, set.cond_list + set.n_cond_list);
    B->set.cond_list = nullptr;
    auto fail = [&](int rc, int i) {
        if (bad_member) *bad_member = i;
        free_batch(B);
        delete B;
        return rc;
    };

    // host preparation of every member (validation first, so that malformed
    // input is rejected without a device); lanes per row are chosen for the
    // smallest team (one 256-thread CTA, 8 warps) so that any mapping can run
    const long long warps = 8;
    B->mem.resize(count);
    std::vector<int> mat_of(count, -1);
    for (int i = 0; i < count; ++i) {
        const acs_instance& I = members[i];
        Member& M = B->mem[i];
        if (I.share_A_with >= 0) {
            const int j = I.share_A_with;
            if (j >= i || I.m != members[j].m || I.n != members[j].n) return fail(ACS_ERR_ARG, i);
            int root = j;                                // the member that holds the data
            while (members[root].share_A_with >= 0) root = members[root].share_A_with;
            const int rc = host::validate(I.m, I.n, members[root].row_ptr, members[root].col, members[root].val,
                                          I.b, I.c, I.n_orthant, I.n_soc, I.soc_dims);
            if (rc != ACS_SOLVED) return fail(rc, i);
            mat_of[i] = mat_of[j];
        } else {
            if (I.share_A_with < -1) return fail(ACS_ERR_ARG, i);
            const int rc = host::validate(I.m, I.n, I.row_ptr, I.col, I.val, I.b, I.c, I.n_orthant, I.n_soc,
                                          I.soc_dims);
            if (rc != ACS_SOLVED) return fail(rc, i);
            Matrix X;
            if (host::build(I.m, I.n, I.row_ptr, I.col, I.val, I.b, I.c, I.n_orthant, I.n_soc, I.soc_dims, warps,
                            warps, X.H) != ACS_SOLVED)
                return fail(ACS_ERR_CSR, i);
            X.stored = (long long)X.H.A.col.size();
            mat_of[i] = (int)B->mats.size();
            B->mats.push_back(std::move(X));
        }
        const Matrix& X = B->mats[mat_of[i]];
        M.m = I.m; M.n = I.n; M.n_orth = I.n_orthant; M.n_soc = I.n_soc; M.mat = mat_of[i];
        M.dense = host::dense_mode(set, I.m);
        if (M.dense) B->dense_m2 = std::max(B->dense_m2, (long long)I.m * I.m);
        M.nnz = X.stored;
        M.b.resize(I.m);
        for (int r = 0; r < I.m; ++r) M.b[r] = I.b[X.H.perm[r]];
        M.c.assign(I.c, I.c + I.n);
        M.soc_off.resize(I.n_soc + 1);
        M.soc_off[0] = I.n_orthant;
        for (int k = 0; k < I.n_soc; ++k) M.soc_off[k + 1] = M.soc_off[k] + I.soc_dims[k];
        double bn = 0, cn = 0;
        for (int r = 0; r < I.m; ++r) bn += I.b[r] * I.b[r];
        for (int j = 0; j < I.n; ++j) cn += I.c[j] * I.c[j];
        M.bnorm = sqrt(bn);
        M.cnorm = sqrt(cn);
    }
    // members in decreasing order of work (stored entries of A and A', plus vectors)
    B->order.resize(count);
    std::iota(B->order.begin(), B->order.end(), 0);
    std::stable_sort(B->order.begin(), B->order.end(), [&](int a, int b2) {
        const Member& x = B->mem[a];
        const Member& y = B->mem[b2];
        return 2 * x.nnz + 4LL * (x.m + x.n) > 2 * y.nnz + 4LL * (y.m + y.n);
    });

    // the device is touched only once every member has passed the host checks
    if (cudaSetDevice(B->device) != cudaSuccess) return fail(ACS_ERR_CUDA, -1);
    if (cudaDeviceGetAttribute(&B->nsm, cudaDevAttrMultiProcessorCount, B->device) != cudaSuccess)
        return fail(ACS_ERR_CUDA, -1);
    {
        int bps = 0;                      // the most CTAs any mapping launches: 256-thread ones
        if (occupancy_for(256, &bps) != ACS_SOLVED) return fail(ACS_ERR_CUDA, -1);
        B->max_ctas = B->nsm * bps;
    }
    if (set.cuda_stream) {
        B->stream = (cudaStream_t)set.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(ACS_ERR_CUDA, -1);
        B->own_stream = true;
    }
    if (cudaEventCreate(&B->ev[0]) != cudaSuccess || cudaEventCreate(&B->ev[1]) != cudaSuccess)
        return fail(ACS_ERR_CUDA, -1);
    // device memory: one allocation, static region uploaded from a host image
    Pool dry;
    layout(B, dry);
    if (cudaMalloc(&B->pool, B->total_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ACS_ERR_OOM, -1);
    }
    {
        std::vector<char> img;
        try {
            img.assign(B->static_bytes, 0);
        } catch (...) {
            return fail(ACS_ERR_OOM, -1);
        }
        for (Matrix& X : B->mats) {
            auto put = [&](const host::HostSell& H, const DevSell& D) {
                put_bytes(img, D.sptr, H.sptr.data(), H.sptr.size());
                put_bytes(img, D.slen, H.slen.data(), H.slen.size());
                put_bytes(img, D.col, H.col.data(), H.col.size());
                std::vector<float> f(H.val.size());
                for (size_t k = 0; k < f.size(); ++k) f[k] = (float)H.val[k];
                put_bytes(img, D.v32, f.data(), f.size());
                put_bytes(img, D.v64, H.val.data(), H.val.size());
            };
            put(X.H.A, X.dA);
            put(X.H.AT, X.dAT);
        }
        for (Member& M : B->mem) {
            put_bytes(img, M.db, M.b.data(), M.b.size());
            put_bytes(img, M.dc, M.c.data(), M.c.size());
            put_bytes(img, M.dsoc, M.soc_off.data(), M.soc_off.size());
        }
        put_bytes(img, B->d_cond_list, B->cond_list_host.data(), B->cond_list_host.size());
        put_bytes(img, B->d_order, B->order.data(), B->order.size());
        if (cudaMemcpy(B->pool, img.data(), B->static_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(ACS_ERR_CUDA, -1);
    }
    if (cudaMemsetAsync(B->pool + B->static_bytes, 0, B->total_bytes - B->static_bytes, B->stream) != cudaSuccess ||
        cudaStreamSynchronize(B->stream) != cudaSuccess)
        return fail(ACS_ERR_CUDA, -1);
    // turn the offsets into device addresses
    char* base = B->pool;
    for (Matrix& X : B->mats) {
        auto fin = [&](const host::HostSell& H, const DevSell& D, SellMat& S) {
            S.nrows = H.nrows; S.nslices = H.nslices; S.g = H.g;
            S.sptr = rebase(D.sptr, base); S.slen = rebase(D.slen, base); S.col = rebase(D.col, base);
            S.v32 = rebase(D.v32, base); S.v64 = rebase(D.v64, base);
        };
        fin(X.H.A, X.dA, X.A);
        fin(X.H.AT, X.dAT, X.AT);
    }
    for (Member& M : B->mem) {
        M.db = rebase(M.db, base); M.dc = rebase(M.dc, base); M.dsoc = rebase(M.dsoc, base);
        M.x = rebase(M.x, base); M.z = rebase(M.z, base); M.ocone = rebase(M.ocone, base);
        Outer& X = M.X;
        X.s = rebase(X.s, base); X.p = rebase(X.p, base); X.g = rebase(X.g, base); X.q = rebase(X.q, base);
        X.chat = rebase(X.chat, base); X.O = rebase(X.O, base); X.w = rebase(X.w, base);
        X.btil = rebase(X.btil, base);
        auto inner = [&](auto& V) {
            V.r = rebase(V.r, base); V.u = rebase(V.u, base); V.p = rebase(V.p, base); V.sv = rebase(V.sv, base);
            V.au = rebase(V.au, base); V.jinv = rebase(V.jinv, base); V.t = rebase(V.t, base);
            V.O2 = rebase(V.O2, base);
        };
        inner(M.V32);
        inner(M.V64);
    }
    B->d_cond_list = rebase(B->d_cond_list, base);
    B->d_order = rebase(B->d_order, base);
    B->d_p32 = rebase(B->d_p32, base);
    B->d_p64 = rebase(B->d_p64, base);
    B->d_ctl = rebase(B->d_ctl, base);
    B->d_head = rebase(B->d_head, base);
    B->d_mailbox = rebase(B->d_mailbox, base);
    B->d_team_bar = rebase(B->d_team_bar, base);
    B->d_team_part = rebase(B->d_team_part, base);
    B->d_team_err = rebase(B->d_team_err, base);
    B->d_dense = rebase(B->d_dense, base);
    // the host images are no longer needed (keep the row relabelling)
    for (Matrix& X : B->mats) {
        std::vector<int> perm = std::move(X.H.perm);
        X.H = host::HostProblem();
        X.H.perm = std::move(perm);
    }
    const int rc = set_mapping(B, map0);
    if (rc != ACS_SOLVED) return fail(rc, -1);
    *out = reinterpret_cast<acs_batch*>(B);
    return ACS_SOLVED;
}

int acs_batch_set_mapping(acs_batch* h, const acs_batch_mapping* mapping) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || !mapping) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    return acs::set_mapping(B, *mapping);
}

int acs_batch_solve_async(acs_batch* h, double tol, int32_t max_iter) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || !(tol >= 0) || max_iter < 0) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    return acs::launch(B, tol, max_iter, true);
}

int acs_batch_results(acs_batch* h, int32_t* status, int32_t* iters, double* residuals) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    if (acs::fetch_controls(B) != ACS_SOLVED) return ACS_ERR_CUDA;
    int worst = ACS_SOLVED;
    for (int i = 0; i < B->count; ++i) {
        const acs::Control& C = B->ctl_host[i];
        const int s = acs::member_status(C);
        if (status) status[i] = s;
        if (iters) iters[i] = C.l;
        if (residuals) {
            for (int k = 0; k < 6; ++k) residuals[8 * i + k] = C.res[k];
            residuals[8 * i + 6] = (double)C.cg_iters;
            residuals[8 * i + 7] = (double)C.switched_at;
        }
        if (s < 0 && worst >= 0) worst = s;
        else if (s == ACS_MAX_ITER && worst == ACS_SOLVED) worst = ACS_MAX_ITER;
    }
    return worst;
}

int acs_batch_solve(acs_batch* h, double tol, int32_t max_iter) {
    const int rc = acs_batch_solve_async(h, tol, max_iter);
    if (rc != ACS_SOLVED) return rc;
    return acs_batch_results(h, nullptr, nullptr, nullptr);
}

int acs_batch_get(acs_batch* h, int32_t i, double* x, double* y, double* s, int32_t* iters, double* residuals) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || i < 0 || i >= B->count) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    const acs::Member& M = B->mem[i];
    acs::Control C;
    cudaStream_t st = B->stream;
    std::vector<double> w;
    if (cudaMemcpyAsync(&C, B->d_ctl + i, sizeof(C), cudaMemcpyDeviceToHost, st) != cudaSuccess) return ACS_ERR_CUDA;
    if (x && cudaMemcpyAsync(x, M.x, sizeof(double) * M.n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ACS_ERR_CUDA;
    if (s && cudaMemcpyAsync(s, M.z, sizeof(double) * M.n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ACS_ERR_CUDA;
    if (y) {
        w.resize(M.m);
        if (cudaMemcpyAsync(w.data(), M.X.w, sizeof(double) * M.m, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return ACS_ERR_CUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return ACS_ERR_CUDA;
    if (y) {
        const std::vector<int>& perm = B->mats[M.mat].H.perm;
        for (int r = 0; r < M.m; ++r) y[perm[r]] = w[r] / B->set.mu;
    }
    if (iters) *iters = C.l;
    if (residuals) {
        for (int k = 0; k < 6; ++k) residuals[k] = C.res[k];
        residuals[6] = (double)C.cg_iters;
        residuals[7] = (double)C.switched_at;
    }
    return acs::member_status(C);
}

int acs_batch_autotune(acs_batch* h, int32_t max_iter, acs_batch_mapping* chosen, double* ms) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || max_iter <= 0) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    const acs_batch_mapping keep = B->map;
    double best = INFINITY;
    acs_batch_mapping best_map = keep;
    int idx = 0;
    for (int th : acs::kThreadChoices)
        for (int g : acs::kTeamChoices) {
            const acs_batch_mapping cand{th, g};
            double t = -1.0;
            if (acs::set_mapping(B, cand) == ACS_SOLVED) {
                // one untimed run (warms caches and the launch), then a timed one
                int rc = acs::launch(B, 0.0, max_iter, false);
                if (rc == ACS_SOLVED) rc = acs::launch(B, 0.0, max_iter, false);
                float f = 0.f;
                if (rc == ACS_SOLVED && cudaEventSynchronize(B->ev[1]) == cudaSuccess &&
                    cudaEventElapsedTime(&f, B->ev[0], B->ev[1]) == cudaSuccess) {
                    t = f;
                    if (t < best) { best = t; best_map = cand; }
                }
            }
            if (ms) ms[idx] = t;
            ++idx;
        }
    if (!(best < INFINITY)) {
        acs::set_mapping(B, keep);
        return ACS_ERR_CUDA;
    }
    const int rc = acs::set_mapping(B, best_map);
    if (chosen) *chosen = best_map;
    return rc;
}

int acs_batch_last_ms(acs_batch* h, double* ms) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || !ms) return ACS_ERR_ARG;
    float f = 0.f;
    if (cudaEventSynchronize(B->ev[1]) != cudaSuccess || cudaEventElapsedTime(&f, B->ev[0], B->ev[1]) != cudaSuccess)
        return ACS_ERR_CUDA;
    *ms = (double)f;
    return ACS_SOLVED;
}

int acs_batch_info(acs_batch* h, long long* out8, long long* counters6) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || !out8) return ACS_ERR_ARG;
    long long sm = 0, sn = 0, nnz = 0;
    for (const auto& M : B->mem) { sm += M.m; sn += M.n; }
    for (const auto& X : B->mats) nnz += X.stored;
    out8[0] = B->count;
    out8[1] = (long long)B->mats.size();
    out8[2] = sm;
    out8[3] = sn;
    out8[4] = nnz;
    out8[5] = B->grid / B->map.team_ctas;
    out8[6] = B->grid;
    out8[7] = B->last_graph ? 1 : 0;
    if (counters6) {
        if (acs::fetch_controls(B) != ACS_SOLVED) return ACS_ERR_CUDA;
        for (int k = 0; k < 6; ++k) counters6[k] = 0;
        for (const auto& C : B->ctl_host) {
            counters6[0] += C.n_cg_A; counters6[1] += C.n_cg_AT; counters6[2] += C.n_64_A;
            counters6[3] += C.n_64_AT; counters6[4] += C.n_cond; counters6[5] += C.n_checks;
        }
    }
    return ACS_SOLVED;
}

int acs_batch_counters(acs_batch* h, long long* out) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || !out) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    if (acs::fetch_controls(B) != ACS_SOLVED) return ACS_ERR_CUDA;
    for (int i = 0; i < B->count; ++i) {
        const acs::Control& C = B->ctl_host[i];
        long long* o = out + 8 * (size_t)i;
        o[0] = C.n_cg_A; o[1] = C.n_cg_AT; o[2] = C.n_64_A; o[3] = C.n_64_AT;
        o[4] = C.n_cond; o[5] = C.n_checks; o[6] = C.n_dense_solve; o[7] = C.n_dense_factor;
    }
    return ACS_SOLVED;
}

int acs_batch_member_ms(acs_batch* h, double* ms) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || !ms) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    if (acs::fetch_controls(B) != ACS_SOLVED) return ACS_ERR_CUDA;
    for (int i = 0; i < B->count; ++i) {
        unsigned long long t = 0;
        for (int k = 0; k < acs::PH_COUNT; ++k) t += B->ctl_host[i].phase_ns[k];
        ms[i] = (double)t * 1e-6;
    }
    return ACS_SOLVED;
}

void acs_batch_destroy(acs_batch* h) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B) return;
    cudaSetDevice(B->device);
    if (B->stream) cudaStreamSynchronize(B->stream);
    acs::free_batch(B);
    delete B;
}

}  // extern "C"
