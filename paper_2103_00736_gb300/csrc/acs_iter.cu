// Persistent iteration kernel of the adaptive-conditioning conic solver.
//
// One cooperative launch runs Algorithm 2 (arXiv 2103.00736, Section IV)
// until the KKT test passes or the iteration limit is reached.  Work inside
// the launch is split into phases separated by a bounded grid barrier; every
// phase is a grid-stride loop over rows of A, rows of A' (= coordinates), or
// cones.
//
// Precision: the outer iteration (s, p, q, w, c_hat, b_tilde, O, x, z) is
// FP64 and its two matrix passes per iteration use the FP64 values of A.
// The projection solve is a correction solve M dw = r0 with r0 the FP64
// residual of the current w, run by preconditioned CG in precision T (FP32
// by default, FP64 on request) and added to w in FP64: one step of
// mixed-precision iterative refinement per outer iteration, so errors left by
// the FP32 solve are corrected by the next iteration's FP64 residual.
//
// Notation (scaled space of Algorithm 2, A_hat = A O, c_hat = O c):
//   p = abs_K(s)                                     (step 17)
//   w = M^{-1}(b_tilde - A_hat p),  M = A_hat A_hat',  b_tilde = b + mu A_hat c_hat
//   s <- (s + p)/2 - mu c_hat + A_hat' w              (steps 18-19, one-solve form)
//   x = O (p + s)/2,  z = O^{-1}(p - s)/(2 mu),  y = w/mu   (steps 20-21)
// The one-solve form follows from abs_A(v) = 2 A_hat' M^{-1} A_hat v - v and
// d = A_hat' M^{-1} b + (mu/2)(abs_A(c_hat) - c_hat) = A_hat' M^{-1} b_tilde - mu c_hat.
// A_hat is never formed: A_hat v = A (O v) and A_hat' u = O (A' u), so the
// rescaling of step 12 costs nothing in the matrix passes.
//
// The projection solve warm-starts from the previous w.  Its initial
// residual b_tilde - M w = b_tilde - A_hat (p + q) with q = A_hat' w from the
// previous update, so no extra matrix pass is needed for the warm start.
//
// Inexact projection: CG stops once sqrt(r' J^{-1} r), an estimate of the
// energy-norm error ||A_hat'(w - w_exact)|| = error of q, is below
// max(eta ||s_l - s_{l-1}||, tol_abs ||s_l||, relfloor sqrt(r0' J^{-1} r0)):
// the projection error is kept a fixed fraction eta of the current step, so it
// vanishes as the iteration converges (a relative inexactness rule).

#include "acs_cbsell.cuh"
#include "acs_device.cuh"
#include "acs_host.cuh"

namespace acs {

// Barrier latency probe: n grid_syncs with one reduced value each.  With
// absent >= 0 that CTA never arrives (the failure-path test): the others'
// bounded waits run out, record ACS_ERR_DEVICE_TIMEOUT and leave; no trap.
__global__ void __launch_bounds__(kThreads, 1)
barrier_probe_kernel(Control* ctl, unsigned* flags, double* partials, int n, double* out, int absent) {
    if ((int)blockIdx.x == absent) return;
    team_set(blockIdx.x, gridDim.x, &ctl->bar_count64, partials);
    sync_init(ctl->bar_gen);
    const unsigned long long t0 = gtimer();
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
        const double v[1] = {1.0};
        const int op[1] = {0};
        block_partials<1>(v, op, partials);
        if (!grid_sync(&ctl->err)) break;
        double r[1];
        grid_combine<1>(partials, op, r);
        acc += r[0];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[0] = (double)(gtimer() - t0) / n;
        out[1] = acc;
        ctl->bar_gen = sync_smem().gen;
    }
}

// Pass micro-benchmark: `reps` repetitions of one kind of phase of the
// persistent kernel on a prepared problem, each followed by a grid barrier,
// timed by CTA 0 on the device's global timer.  Kinds: 0 column-blocked A'
// pass (partial sums of A'u), 1 combine t = O^2 A'u and u'Mu, 2 column-
// blocked A pass, 3 CG vector step combining its partial sums, 4 / 5 / 6 the
// same three on the L2-gather layout (FP32 values), 7 FP64 projection
// residual pass over A, 8 FP64 pass over A' (q = A_hat' w), 9 the barrier
// alone, 10 abs_K, 11 KKT residuals, 12 / 13 FP32 outer projection residual
// (pass, combine), 14 / 15 FP32 outer update (pass, combine), 16 / 17 the
// staging of the column-blocked A pass alone (FP32 / FP64 source), 18 the
// column-blocked A' pass without its gathers, 19 without its staging, 20 / 21
// the CTA's entries of the A' image as a plain linear stream (columns and
// values / values only).  Phases whose
// layout the problem lacks do nothing.  The iterate state of the problem is
// left undefined (the next acs_solve starts afresh unless acs_set_state).
__global__ void __launch_bounds__(kThreads, 1)
pass_bench_kernel(const __grid_constant__ IterParams<float> P, const __grid_constant__ IterParams<double> P64, int kind,
                  int reps, double* out_ns) {
    team_set(blockIdx.x, gridDim.x, &P.ctl->bar_count64, P.partials);
    sync_init(P.ctl->bar_gen);
    if (P.Acb.nblocks > 0) cb_init();
    const bool cbA = P.Acb.nblocks > 0, cbT = P.ATcb.nblocks > 0;
    const bool l2A = P.A.v32 != nullptr, l2T = P.AT.v32 != nullptr;
    const unsigned long long t0 = gtimer();
    int r = 0;
    for (; r < reps; ++r) {
        switch (kind) {
            case 0: if (cbT) phase_cg_At_cb(P); break;
            case 1: if (cbT) phase_cg_tcomb(P); break;
            case 2: if (cbA) phase_cg_A_cb(P); break;
            case 3: if (cbA) phase_cg_vec<float, true>(P, 0.0, 0.f); break;
            case 4: if (l2T) phase_cg_At(P); break;
            case 5: if (l2A) phase_cg_A(P); break;
            case 6: if (l2A) phase_cg_vec<float, false>(P, 0.0, 0.f); break;
            case 7: phase_rhs(P64); break;
            case 8: phase_update(P64, false, false); break;
            case 10: phase_abs(P64, 0.0); break;
            case 11: phase_kkt(P64); break;
            case 12: if (cbA) phase_rhs_cb(P); break;
            case 13: if (cbA) phase_rhs_comb(P); break;
            case 14: if (cbT) phase_update_cb(P); break;
            case 15: if (cbT) phase_update_comb(P, false); break;
            case 16: if (cbA) cb_stage_only(P.Acb, P.V.t, &P.ctl->err); break;
            case 17: if (cbA) cb_stage_only(P.Acb, P.X.g, &P.ctl->err); break;
            case 18: if (cbT) cb_pass<float, 1>(P.ATcb, P.V.u, &P.ctl->err); break;
            case 19: if (cbT) cb_pass<float, 2>(P.ATcb, P.V.u, &P.ctl->err); break;
            case 20: if (cbT) cb_pass<float, 3>(P.ATcb, P.V.u, &P.ctl->err); break;
            case 21: if (cbT) cb_pass<float, 4>(P.ATcb, P.V.u, &P.ctl->err); break;
            default: break;
        }
        if (!grid_sync(&P.ctl->err)) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out_ns[0] = r == reps ? (double)(gtimer() - t0) / reps : -1.0;
        P.ctl->bar_gen = sync_smem().gen;
    }
}

// ---------------------------------------------------------------------------
// the persistent single-problem kernel: one team = the whole grid
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) iter_kernel(const __grid_constant__ IterParams<T> P) {
    const int status0 = ld_volatile_int(&P.ctl->status);
    // the FP32 launch runs from a fresh or resumed state; the FP64 launch of a
    // mixed-precision solve runs only if the FP32 launch handed over
    if (sizeof(T) == 4 ? status0 != ST_RUNNING : (status0 != ST_RUNNING && status0 != ST_SWITCH)) return;
    team_set(blockIdx.x, gridDim.x, &P.ctl->bar_count64, P.partials, P.dense ? P.dM : nullptr,
             P.dense ? P.dX : nullptr);
    sync_init(P.ctl->bar_gen);
    if (P.Acb.nblocks > 0) cb_init();
    solve_loop<T>(P, status0);
}

// LP crossover polish of the current iterate (FP64; see polish_loop).
__global__ void __launch_bounds__(kThreads, 1) polish_kernel(const __grid_constant__ IterParams<double> P,
                                                             const __grid_constant__ IterParams<float> P32,
                                                             const __grid_constant__ IterParams<double> Q,
                                                             const PolishOut out, int rounds, double rel,
                                                             int fp32) {
    team_set(blockIdx.x, gridDim.x, &P.ctl->bar_count64, P.partials, P.dM, P.dX);
    sync_init(P.ctl->bar_gen);
    polish_loop(P, P32, Q, out, rounds, rel, fp32 != 0);
}

// ---------------------------------------------------------------------------
// small setup kernels used by the solve
// ---------------------------------------------------------------------------

// the grid barrier's counters, restarted for a launch outside a solve
__global__ void reset_barrier(Control* ctl) {
    ctl->bar_count = 0;
    ctl->bar_gen = 0;
    ctl->bar_count64 = 0;
}

__global__ void init_zero_kernel(double* x, double* z, double* w, double* q, int n, int m) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        x[j] = 0.0;
        z[j] = 0.0;
        q[j] = 0.0;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) w[i] = 0.0;
}
__global__ void init_identity_heads(double* x, double* z, int n_orth, const int* soc_off, int n_soc) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n_orth) { x[j] = 1.0; z[j] = 1.0; }
    if (j < n_soc) { const int a = soc_off[j]; x[a] = 1.0; z[a] = 1.0; }
}
__global__ void reset_flags(unsigned* flags, unsigned* release, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) flags[i] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) *release = 0u;
}
__global__ void reset_control(Control* ctl, int l, double ds, double snorm, double eta) {
    ctl->status = ST_RUNNING;
    ctl->err = 0;
    ctl->l = l;
    ctl->cg_iters = 0;
    ctl->switched_at = 0;
    for (int i = 0; i < 6; ++i) ctl->res[i] = NAN;
    ctl->ds = ds;
    ctl->snorm = snorm;
    ctl->eta = eta;
    ctl->n_cg_A = ctl->n_cg_AT = ctl->n_64_A = ctl->n_64_AT = ctl->n_cond = ctl->n_checks = 0;
    for (int i = 0; i < PH_COUNT; ++i) { ctl->phase_ns[i] = 0; ctl->phase_n[i] = 0; }
    ctl->bar_count = 0;
    ctl->bar_gen = 0;
    ctl->bar_count64 = 0;
    ctl->stage = 0;
    ctl->dense_on = 0;
    ctl->dense_failed = 0;
    ctl->win_it = 0;
    ctl->win_cg = 0;
    ctl->extrap_ok = 0;
    ctl->factor_ok = 0;
    ctl->n_dense_solve = ctl->n_dense_factor = 0;
    ctl->n_32_A = ctl->n_32_AT = 0;
    ctl->outer32_end = 0;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <typename T>
static IterParams<T> make_params(Problem* P, double tol, int max_iter, const Inner<T>& V) {
    IterParams<T> Q{};
    Q.m = P->m; Q.n = P->n; Q.n_orth = P->n_orth; Q.n_soc = P->n_soc;
    Q.A = P->A; Q.AT = P->AT;
    Q.soc_off = P->soc_off;
    Q.b = P->b; Q.c = P->c; Q.bnorm = P->bnorm; Q.cnorm = P->cnorm;
    Q.X = P->X;
    Q.V = V;
    Q.x = P->x; Q.z = P->z; Q.ocone = P->ocone;
    Q.partials = P->partials;
    Q.flags = P->flags; Q.release = P->release; Q.bcast = P->bcast;
    Q.ctl = P->ctl;
    Q.mu = P->set.mu; Q.t_cond = P->set.t;
    Q.cond_first = P->set.cond_first; Q.cond_period = P->set.cond_period;
    Q.cond_list = P->cond_list; Q.n_cond_list = (int)P->cond_list_host.size();
    Q.check_every = P->set.check_every > 0 ? P->set.check_every : 1;
    Q.max_iter = max_iter;
    Q.tol = tol;
    Q.cg_eta = P->set.cg_eta;
    Q.cg_tol = P->set.cg_tol;
    Q.cg_relfloor = sizeof(T) == 4 ? 1e-6 : 1e-13;
    Q.cg_max = P->set.cg_max_iter;
    Q.refresh = P->warm ? 1 : 0;
    Q.refine = P->set.cg_refine > 0 ? P->set.cg_refine : 1;
    Q.switch_ok = P->set.precision != ACS_PREC_FP64 ? 1 : 0;
    Q.dense = P->dense;
    Q.switch_budget = acs::host::switch_budget(P->set, P->m, P->padded_A, P->full_rows);
    Q.extrap = P->set.extrapolation;
    Q.admm = P->set.splitting == ACS_SPLIT_ADMM ? 1 : 0;
    Q.full_rows = P->full_rows ? 1 : 0;
    Q.dM = P->dM;
    Q.dX = P->dX;
    if (sizeof(T) == 4) {                 // column-blocked passes: FP32 loop only
        Q.Acb = P->Acb;
        Q.ATcb = P->ATcb;
        Q.outer32 = P->set.precision == ACS_PREC_FP32 && P->Acb.nblocks > 0 ? 1 : 0;
        Q.outer32_tol = P->set.outer32_tol;
        Q.outer32_l2 = P->outer_f32 ? 1 : 0;
    }
    return Q;
}

// Dynamic shared memory the FP32 launch may ask for: one block of a
// column-blocked pass (the block width limit in FP32 entries).
int cb_smem_limit() { return kCbMaxWidth * (int)sizeof(float); }

int occupancy_grid(Problem* P) {
    int nsm = 0, b32 = 0, b64 = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess)
        return ACS_ERR_CUDA;
    // the FP32 launch is sized with the largest block it may stage, so that
    // the grid (and the ranges of items dealt to its CTAs) does not depend on
    // the block width chosen later
    if (cudaFuncSetAttribute(iter_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, cb_smem_limit()) !=
        cudaSuccess)
        return ACS_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, iter_kernel<float>, kThreads, cb_smem_limit()) !=
        cudaSuccess)
        return ACS_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, iter_kernel<double>, kThreads, 0) != cudaSuccess)
        return ACS_ERR_CUDA;
    if (b32 < 1 || b64 < 1) return ACS_ERR_CUDA;
    P->grid32 = nsm * b32;
    P->grid64 = nsm * b64;
    return ACS_SOLVED;
}

template <typename T>
static cudaError_t launch_iter(Problem* P, const IterParams<T>& Q, int grid) {
    void* args[] = {(void*)&Q};
    const size_t smem = sizeof(T) == 4 ? (size_t)P->cb_smem : 0;
    return cudaLaunchCooperativeKernel((const void*)iter_kernel<T>, dim3(grid), dim3(kThreads), args, smem,
                                       P->stream);
}

int pass_bench(Problem* P, int kind, int reps, int smem_bytes, double* us) {
    // the stream-only variant (18) reads no shared memory: any size may be asked for
    const int need = (kind == 18 || kind == 20 || kind == 21) ? 0 : P->cb_smem;
    if (smem_bytes < need || smem_bytes > cb_smem_limit() || reps <= 0) return ACS_ERR_ARG;
    cudaStream_t st = P->stream;
    if (cudaFuncSetAttribute(pass_bench_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cb_smem_limit()) !=
        cudaSuccess)
        return ACS_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pass_bench_kernel, kThreads, smem_bytes) !=
            cudaSuccess ||
        per_sm < 1)
        return ACS_ERR_CUDA;
    reset_flags<<<1, 256, 0, st>>>(P->flags, P->release, P->max_ctas);
    reset_control<<<1, 1, 0, st>>>(P->ctl, 0, INFINITY, 0.0, P->set.cg_eta);
    IterParams<float> Q = make_params<float>(P, 0.0, 1, P->V32);
    IterParams<double> Q64 = make_params<double>(P, 0.0, 1, P->V64);
    double* d_out = P->bcast;
    void* args[] = {(void*)&Q, (void*)&Q64, (void*)&kind, (void*)&reps, (void*)&d_out};
    // the grid the column-blocked ranges were dealt to
    if (cudaLaunchCooperativeKernel((const void*)pass_bench_kernel, dim3(P->grid32), dim3(kThreads), args,
                                    (size_t)smem_bytes, st) != cudaSuccess)
        return ACS_ERR_CUDA;
    double h = 0.0;
    int err = 0;
    if (cudaMemcpyAsync(&h, d_out, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&err, &P->ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ACS_ERR_CUDA;
    if (err != 0) return err;
    *us = h * 1e-3;
    return ACS_SOLVED;
}

int barrier_probe(Problem* P, int n, double* ns_per_barrier, int absent) {
    cudaStream_t st = P->stream;
    reset_flags<<<1, 256, 0, st>>>(P->flags, P->release, P->max_ctas);
    reset_control<<<1, 1, 0, st>>>(P->ctl, 0, INFINITY, 0.0, P->set.cg_eta);
    double* d_out = P->bcast;
    void* args[] = {(void*)&P->ctl, (void*)&P->flags, (void*)&P->partials, (void*)&n, (void*)&d_out,
                    (void*)&absent};
    if (cudaLaunchCooperativeKernel((const void*)barrier_probe_kernel, dim3(P->grid32), dim3(kThreads), args, 0,
                                    st) != cudaSuccess)
        return ACS_ERR_CUDA;
    double h[2];
    int err = 0;
    if (cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&err, &P->ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ACS_ERR_CUDA;
    *ns_per_barrier = h[0];
    if (err != 0) return err;
    if (h[1] != (double)n * P->grid32 * kThreads) return ACS_ERR_DEVICE_TIMEOUT;
    return ACS_SOLVED;
}

int launch_polish(Problem* P, int rounds, double rel) {
    cudaStream_t st = P->stream;
    const int n = P->n, m = P->m;
    if (!P->px) {
        // owned by the problem from here on (released with it, also if a later one fails)
        if (!P->alloc(&P->px, n) || !P->alloc(&P->pw, m) || !P->alloc(&P->pz, n) || !P->alloc(&P->pwork, m) ||
            !P->alloc(&P->pres, 16)) {
            P->px = nullptr;
            return ACS_ERR_OOM;
        }
    }
    // the factored M = A_B A_B' (m <= kDenseLimit): the handle's cached-
    // operator scratch, else the polish's own
    double *dM = P->dM, *dX = P->dX;
    if (!dM && m <= (P->full_rows ? host::kDenseRowsLimit : host::kDenseLimit)) {
        if (!P->pdM) {
            if (!P->alloc(&P->pdM, (size_t)m * m) || !P->alloc(&P->pdX, (size_t)m * m)) {
                P->pdM = P->pdX = nullptr;
                return ACS_ERR_OOM;
            }
        }
        dM = P->pdM;
        dX = P->pdX;
    }
    if (cudaMemcpyAsync(P->pw, P->X.w, sizeof(double) * m, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(P->pres, 0, sizeof(double) * 16, st) != cudaSuccess)
        return ACS_ERR_CUDA;
    reset_barrier<<<1, 1, 0, st>>>(P->ctl);
    if (cudaGetLastError() != cudaSuccess) return ACS_ERR_CUDA;
    IterParams<double> Q = make_params<double>(P, 0.0, 1, P->V64);
    Q.dense = 0;
    Q.X.w = P->pwork;                     // the solves' w: the iterate's w stays
    Q.dM = dM;
    Q.dX = dX;
    IterParams<double> Qk = Q;            // the residuals of the polished point: all of A
    // the corrections by FP32 CG (refined by FP64 rounds) when the target
    // leaves room for it, on the problem's FP32 values
    int fp32 = !dM && rel > 1e-10 && P->A.v32 && P->AT.v32 ? 1 : 0;
    IterParams<float> Q32 = make_params<float>(P, 0.0, 1, P->V32);
    Q32.dense = 0;
    Q32.X.w = P->pwork;
    Q32.Acb.nblocks = Q32.ATcb.nblocks = 0;
    Q32.outer32 = 0;
    if (!dM) {
        // CG corrections: the passes over the rows of A run on A_B, the rows of
        // A restricted to the support's columns (the other columns carry
        // O_j = 0); those over A' skip the rows off the support
        SellMat AB;
        const int rc = support_rows(P, AB, fp32 != 0);
        if (rc != ACS_SOLVED) return rc;
        Q.A = AB;
        Q.full_rows = 0;
        Q32.A = AB;
        Q32.full_rows = 0;
    }
    Qk.x = P->px;
    Qk.z = P->pz;
    Qk.X.w = P->pw;
    PolishOut out{P->px, P->pw, P->pz, P->pres, P->pres + 8};
    void* args[] = {(void*)&Q, (void*)&Q32, (void*)&Qk, (void*)&out, (void*)&rounds, (void*)&rel, (void*)&fp32};
    if (cudaLaunchCooperativeKernel((const void*)polish_kernel, dim3(P->grid64), dim3(kThreads), args, 0, st) !=
        cudaSuccess)
        return ACS_ERR_CUDA;
    return ACS_SOLVED;
}

int launch_solve(Problem* P, double tol, int max_iter) {
    cudaStream_t st = P->stream;
    const int n = P->n, m = P->m;
    const int big = n > m ? n : m;
    const int nb = (big + 255) / 256 > 4096 ? 4096 : (big + 255) / 256;
    reset_flags<<<1, 256, 0, st>>>(P->flags, P->release, P->max_ctas);
    if (P->warm) reset_control<<<1, 1, 0, st>>>(P->ctl, P->warm_l, P->warm_ds, P->warm_snorm, P->warm_eta);
    else reset_control<<<1, 1, 0, st>>>(P->ctl, 0, INFINITY, 0.0, P->set.cg_eta);
    if (!P->warm) {
        init_zero_kernel<<<nb, 256, 0, st>>>(P->x, P->z, P->X.w, P->X.q, n, m);
        const int h = P->n_orth > P->n_soc ? P->n_orth : P->n_soc;
        if (h > 0) init_identity_heads<<<(h + 255) / 256, 256, 0, st>>>(P->x, P->z, P->n_orth, P->soc_off, P->n_soc);
    }
    if (cudaGetLastError() != cudaSuccess) return ACS_ERR_CUDA;
    cudaError_t e;
    if (P->ev_launch[0]) cudaEventRecord(P->ev_launch[0], st);
    if (P->set.precision == ACS_PREC_FP64 || P->dense == 1) {
        // the cached operator runs in the FP64 loop (exact corrections)
        IterParams<double> Q = make_params<double>(P, tol, max_iter, P->V64);
        e = launch_iter<double>(P, Q, P->grid64);
    } else {
        IterParams<float> Q = make_params<float>(P, tol, max_iter, P->V32);
        e = launch_iter<float>(P, Q, P->grid32);
        if (e == cudaSuccess) {
            // continues only if the FP32 solve handed over (returns at once otherwise)
            IterParams<double> Q64 = make_params<double>(P, tol, max_iter, P->V64);
            Q64.refresh = 0;
            e = launch_iter<double>(P, Q64, P->grid64);
        }
    }
    if (P->ev_launch[1]) cudaEventRecord(P->ev_launch[1], st);
    P->warm = false;
    P->state_clobbered = false;
    ++P->solves;
    if (e != cudaSuccess) {
        fprintf(stderr, "acs: cooperative launch failed: %s\n", cudaGetErrorString(e));
        return ACS_ERR_CUDA;
    }
    return ACS_SOLVED;
}

}  // namespace acs
