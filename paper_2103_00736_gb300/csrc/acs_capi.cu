// C ABI of the conic solver: problem creation (validation, transpose, upload),
// solve, result and state transfer, destruction.  See include/acs.h.

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>

#include <algorithm>
#include <climits>
#include <new>
#include <vector>

#include "acs_cbsell.cuh"
#include "acs_host.cuh"
#include "acs_internal.cuh"

using acs::Problem;
using acs::host::HostSell;
using acs::host::finite_all;

namespace {

constexpr const char* kVersion = "acs-gb300 0.1 (sm_103a)";

template <typename T>
int dalloc(Problem* P, T** ptr, size_t count) {
    return P->alloc(ptr, count) ? ACS_SOLVED : ACS_ERR_OOM;
}

template <typename T>
int upload(Problem* P, T* dst, const T* src, size_t count) {
    if (count == 0) return ACS_SOLVED;
    if (cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, P->stream) != cudaSuccess)
        return ACS_ERR_CUDA;
    P->h2d_bytes += (long long)(count * sizeof(T));
    return ACS_SOLVED;
}

// The narrow copies of the uploaded FP64 values, on the device: FP32 by the
// conversion's round-to-nearest, BF16 as the upper half of the FP32 value
// rounded to nearest even (the same bit rule as the host's to_bf16).
__global__ void narrow_f32(const double* __restrict__ v64, float* __restrict__ v32, long long tot) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x)
        v32[k] = (float)v64[k];
}
__global__ void narrow_bf16(const double* __restrict__ v64, unsigned short* __restrict__ v16, long long tot) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x) {
        unsigned u = __float_as_uint((float)v64[k]);
        u += 0x7FFFu + ((u >> 16) & 1u);
        v16[k] = (unsigned short)(u >> 16);
    }
}

// FP64 values always; for the FP32 correction CG either FP32 values or,
// with BF16 storage of A, BF16 bit patterns (v32 is then NULL).  narrow =
// false: no FP32 copy (the FP32 passes use the column-blocked image).
int upload_sell(Problem* P, const HostSell& H, acs::SellMat& M, bool narrow = true) {
    int* sptr = nullptr; int* slen = nullptr; int* col = nullptr;
    float* v32 = nullptr; double* v64 = nullptr; unsigned short* v16 = nullptr;
    const size_t tot = H.col.size();
    const bool bf16 = P->set.a_storage == ACS_STORE_BF16;
    if (dalloc(P, &sptr, H.sptr.size()) || dalloc(P, &slen, H.slen.size()) || dalloc(P, &col, tot) ||
        (narrow && (bf16 ? dalloc(P, &v16, tot) : dalloc(P, &v32, tot))) || dalloc(P, &v64, tot))
        return ACS_ERR_OOM;
    int rc = 0;
    rc |= upload(P, sptr, H.sptr.data(), H.sptr.size());
    rc |= upload(P, slen, H.slen.data(), H.slen.size());
    rc |= upload(P, col, H.col.data(), tot);
    rc |= upload(P, v64, H.val.data(), tot);
    // the narrow copy of the values, converted on the device from the FP64 upload
    if (narrow && tot > 0) {
        const long long nb = std::min<long long>(((long long)tot + 255) / 256, 4096);
        if (bf16) narrow_bf16<<<(unsigned)nb, 256, 0, P->stream>>>(v64, v16, (long long)tot);
        else narrow_f32<<<(unsigned)nb, 256, 0, P->stream>>>(v64, v32, (long long)tot);
        rc |= cudaGetLastError() != cudaSuccess;
    }
    // the pageable source buffers are released when this function returns
    if (rc || cudaStreamSynchronize(P->stream) != cudaSuccess) return ACS_ERR_CUDA;
    M.nrows = H.nrows; M.nslices = H.nslices; M.g = H.g;
    M.sptr = sptr; M.slen = slen; M.col = col; M.v32 = v32; M.v64 = v64; M.v16 = v16;
    return ACS_SOLVED;
}

// A device-built image (acs_devbuild.cu): its slice tables uploaded and the
// narrow copy of the values converted from the FP64 ones.
int adopt_device_sell(Problem* P, int nrows, int g, const std::vector<int>& sptr_h, const std::vector<int>& slen_h,
                      int* col, double* v64, long long tot, acs::SellMat& M) {
    int* sptr = nullptr; int* slen = nullptr;
    float* v32 = nullptr; unsigned short* v16 = nullptr;
    const bool bf16 = P->set.a_storage == ACS_STORE_BF16;
    if (dalloc(P, &sptr, sptr_h.size()) || dalloc(P, &slen, slen_h.size()) ||
        (bf16 ? dalloc(P, &v16, (size_t)tot) : dalloc(P, &v32, (size_t)tot)))
        return ACS_ERR_OOM;
    int rc = 0;
    rc |= upload(P, sptr, sptr_h.data(), sptr_h.size());
    rc |= upload(P, slen, slen_h.data(), slen_h.size());
    if (tot > 0) {
        const long long nb = std::min<long long>((tot + 255) / 256, 4096);
        if (bf16) narrow_bf16<<<(unsigned)nb, 256, 0, P->stream>>>(v64, v16, tot);
        else narrow_f32<<<(unsigned)nb, 256, 0, P->stream>>>(v64, v32, tot);
        rc |= cudaGetLastError() != cudaSuccess;
    }
    if (rc || cudaStreamSynchronize(P->stream) != cudaSuccess) return ACS_ERR_CUDA;
    M.nrows = nrows; M.nslices = (int)slen_h.size(); M.g = g;
    M.sptr = sptr; M.slen = slen; M.col = col; M.v32 = v32; M.v64 = v64; M.v16 = v16;
    return ACS_SOLVED;
}

// Column-blocked image: offsets, row ids, 16-bit columns, FP32 values, the
// CTAs' item ranges and the partial-sum buffer.
int upload_cb(Problem* P, const acs::host::HostCb& H, acs::CbMat& M) {
    int* sptr = nullptr; unsigned short* rowid = nullptr; unsigned short* col = nullptr;
    float* val = nullptr; int* cta = nullptr; float* part = nullptr; unsigned* cend = nullptr;
    unsigned short* ipos = nullptr;
    const size_t tot = H.col.size();
    if (dalloc(P, &sptr, H.sptr.size()) || dalloc(P, &rowid, H.rowid.size()) || dalloc(P, &col, tot) ||
        dalloc(P, &ipos, H.ipos.size()) ||
        dalloc(P, &val, tot) || dalloc(P, &cta, H.cta_beg.size()) || dalloc(P, &cend, H.cend.size()) ||
        dalloc(P, &part, (size_t)H.nblocks * H.nsl * 32))
        return ACS_ERR_OOM;
    int rc = 0;
    rc |= upload(P, sptr, H.sptr.data(), H.sptr.size());
    rc |= upload(P, rowid, H.rowid.data(), H.rowid.size());
    rc |= upload(P, col, H.col.data(), tot);
    rc |= upload(P, val, H.val.data(), tot);
    rc |= upload(P, cta, H.cta_beg.data(), H.cta_beg.size());
    rc |= upload(P, cend, H.cend.data(), H.cend.size());
    rc |= upload(P, ipos, H.ipos.data(), H.ipos.size());
    if (rc || cudaStreamSynchronize(P->stream) != cudaSuccess) return ACS_ERR_CUDA;
    M.nrows = H.nrows; M.ncols = H.ncols; M.width = H.width; M.nblocks = H.nblocks; M.nsl = H.nsl;
    M.ctas = (int)H.cta_beg.size() - 1;
    M.sptr = sptr; M.rowid = rowid; M.col = col; M.val = val; M.cta_beg = cta; M.part = part; M.cend = cend;
    M.ipos = ipos;
    return ACS_SOLVED;
}

// Whether acs_solve's FP32 passes use the column-blocked layout: on unless
// switched off, with FP32 storage of A, when the FP32 launch runs CG at all.
bool cb_wanted(const acs_settings& set, int dense) {
    return set.col_block >= 0 && set.a_storage == ACS_STORE_FP32 && dense != 1;
}

template <typename T>
int alloc_inner(Problem* P, acs::Inner<T>& V) {
    const int m = P->m, n = P->n;
    int rc = 0;
    rc |= dalloc(P, &V.r, m); rc |= dalloc(P, &V.u, m); rc |= dalloc(P, &V.p, m);
    rc |= dalloc(P, &V.sv, m); rc |= dalloc(P, &V.au, m); rc |= dalloc(P, &V.t, n);
    rc |= dalloc(P, &V.jinv, m); rc |= dalloc(P, &V.O2, n);
    if (rc) return ACS_ERR_OOM;
    // p and sv are multiplied by beta = 0 on the first CG step: keep them finite
    if (cudaMemsetAsync(V.p, 0, sizeof(T) * m, P->stream) != cudaSuccess ||
        cudaMemsetAsync(V.sv, 0, sizeof(T) * m, P->stream) != cudaSuccess)
        return ACS_ERR_CUDA;
    return ACS_SOLVED;
}
int alloc_outer(Problem* P, acs::Outer& X) {
    const int m = P->m, n = P->n;
    int rc = 0;
    rc |= dalloc(P, &X.s, n); rc |= dalloc(P, &X.p, n); rc |= dalloc(P, &X.g, n);
    rc |= dalloc(P, &X.q, n); rc |= dalloc(P, &X.w, m); rc |= dalloc(P, &X.chat, n);
    rc |= dalloc(P, &X.btil, m); rc |= dalloc(P, &X.O, n);
    rc |= dalloc(P, &X.wp, m); rc |= dalloc(P, &X.qp, n);
    return rc ? ACS_ERR_OOM : ACS_SOLVED;
}

void free_all(Problem* P) {
    if (!P) return;
    if (P->stream) cudaStreamSynchronize(P->stream);    // the blocks go back to the cache idle
    for (auto& a : P->allocations) acs::dev_release(P->device, a.first, a.second);
    P->allocations.clear();
    if (P->ctl_host) cudaFreeHost(P->ctl_host);
    P->ctl_host = nullptr;
    for (auto& ev : P->ev_polish) {
        if (ev) cudaEventDestroy(ev);
        ev = nullptr;
    }
    for (auto& ev : P->ev_launch) {
        if (ev) cudaEventDestroy(ev);
        ev = nullptr;
    }
    if (P->own_stream && P->stream) cudaStreamDestroy(P->stream);
    P->stream = nullptr;
}

// One crossover polish of the current iterate (LP; the iteration state other
// than s, w, x, z is used as scratch).  info7 as documented for acs_polish.
// Returns ACS_SOLVED (the polished point replaced x, y, z and the residual
// record) or ACS_POLISH_KEPT, or an error.  Reads the iterate's residuals
// from ctl_host (filled by acs_get).
int polish_once(Problem* P, int rounds, double rel, double* info7) {
    double before = 0.0;
    for (int i = 0; i < 4; ++i) before = fmax(before, P->ctl_host->res[i]);
    cudaEventRecord(P->ev_polish[0], P->stream);
    int rc = acs::launch_polish(P, rounds, rel);
    if (rc != ACS_SOLVED) return rc;
    cudaEventRecord(P->ev_polish[1], P->stream);
    double h16[16];
    int err = 0;
    if (cudaMemcpyAsync(h16, P->pres, sizeof(h16), cudaMemcpyDeviceToHost, P->stream) != cudaSuccess ||
        cudaMemcpyAsync(&err, &P->ctl->err, sizeof(int), cudaMemcpyDeviceToHost, P->stream) != cudaSuccess ||
        cudaStreamSynchronize(P->stream) != cudaSuccess)
        return ACS_ERR_CUDA;
    if (err != 0) return err;
    if (h16[11] != 1.0) return ACS_ERR_NUMERICAL;
    {
        float f = 0.f;
        if (cudaEventElapsedTime(&f, P->ev_polish[0], P->ev_polish[1]) != cudaSuccess) return ACS_ERR_CUDA;
        P->polish_ms += (double)f;
    }
    double after = 0.0;
    for (int i = 0; i < 4; ++i) after = fmax(after, h16[i]);
    const bool take = after < before;                       // NaN compares false: kept
    if (take) {
        cudaStream_t s = P->stream;
        if (cudaMemcpyAsync(P->x, P->px, sizeof(double) * P->n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(P->z, P->pz, sizeof(double) * P->n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(P->X.w, P->pw, sizeof(double) * P->m, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(&P->ctl->res[0], P->pres, sizeof(double) * 6, cudaMemcpyDeviceToDevice, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return ACS_ERR_CUDA;
        for (int i = 0; i < 6; ++i) P->ctl_host->res[i] = h16[i];
    }
    info7[0] = h16[8];
    info7[1] = h16[9];
    info7[2] = h16[10];
    info7[3] = before;
    info7[4] = after;
    info7[5] = take ? 1.0 : 0.0;
    info7[6] = h16[12];
    ++P->pol.attempts;
    P->pol.taken += take ? 1 : 0;
    P->pol.corrections += (long long)(h16[9] + h16[10]);
    P->pol.factored += h16[12] == 1.0 ? 1 : 0;
    P->pol.support = (long long)h16[8];
    P->pol.support_entries = h16[12] == 1.0 ? 0 : P->padded_B;
    return take ? ACS_SOLVED : ACS_POLISH_KEPT;
}

// Counters of a solve run in segments, added up on the host.
void add_counters(acs::Control& acc, const acs::Control& c) {
    acc.cg_iters += c.cg_iters;
    acc.n_cg_A += c.n_cg_A; acc.n_cg_AT += c.n_cg_AT; acc.n_64_A += c.n_64_A; acc.n_64_AT += c.n_64_AT;
    acc.n_cond += c.n_cond; acc.n_checks += c.n_checks;
    acc.n_dense_solve += c.n_dense_solve; acc.n_dense_factor += c.n_dense_factor;
    acc.n_32_A += c.n_32_A; acc.n_32_AT += c.n_32_AT;
    for (int i = 0; i < acs::PH_COUNT; ++i) {
        acc.phase_ns[i] += c.phase_ns[i];
        acc.phase_n[i] += c.phase_n[i];
    }
}

// acs_solve with polish_tol > tol (LP): iterate until every residual is <=
// the current polish level, polish; done if the polished point meets tol,
// else restore the scaling, resume the iteration from its state (as
// acs_set_state does) and try again at a level ten times lower; the last
// segment runs to tol without a polish.
int solve_polished(Problem* P, double tol, int max_iter) {
    double level = P->set.polish_tol;
    acs::Control acc{};
    P->pol = acs::PolishStats{};
    P->seg_ms = P->polish_ms = 0.0;
    P->polished_solve = true;
    const int n = P->n;
    if (!P->psaveO && dalloc(P, &P->psaveO, (size_t)n)) return ACS_ERR_OOM;
    if (!P->psaveW && dalloc(P, &P->psaveW, (size_t)P->m)) return ACS_ERR_OOM;
    if (!P->psaveX && dalloc(P, &P->psaveX, (size_t)n)) return ACS_ERR_OOM;
    if (!P->psaveZ && dalloc(P, &P->psaveZ, (size_t)n)) return ACS_ERR_OOM;
    int st = ACS_ERR_CUDA;
    for (;;) {
        const double target = fmax(tol, level);
        // a segment that ends at a polish level runs its outer products in
        // FP32 (the polish, not the iteration, sets the final accuracy); the
        // last segment, to tol itself, in FP64
        P->outer_f32 = target > tol;
        int rc = acs::launch_solve(P, target, max_iter);
        P->outer_f32 = false;
        if (rc != ACS_SOLVED) return rc;
        if (cudaMemcpyAsync(P->ctl_host, P->ctl, sizeof(acs::Control), cudaMemcpyDeviceToHost, P->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(P->stream) != cudaSuccess)
            return ACS_ERR_CUDA;
        add_counters(acc, *P->ctl_host);
        {
            float f = 0.f;
            if (cudaEventElapsedTime(&f, P->ev_launch[0], P->ev_launch[1]) != cudaSuccess) return ACS_ERR_CUDA;
            P->seg_ms += (double)f;
        }
        st = P->ctl_host->status;
        if (st == acs::ST_RUNNING || st == acs::ST_SWITCH) st = ACS_ERR_CUDA;
        if (st != ACS_SOLVED || target <= tol) break;
        const acs::Control seg = *P->ctl_host;
        if (cudaMemcpyAsync(P->psaveO, P->X.O, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(P->psaveW, P->X.w, sizeof(double) * P->m, cudaMemcpyDeviceToDevice, P->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(P->psaveX, P->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream) != cudaSuccess ||
            cudaMemcpyAsync(P->psaveZ, P->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream) != cudaSuccess)
            return ACS_ERR_CUDA;
        // the polished point need only meet tol: its solves stop at 1e-3 tol /
        // polish_tol of their first residual (the iterate's, about polish_tol)
        double info[7];
        rc = polish_once(P, 3, fmax(1e-13, 1e-3 * tol / P->set.polish_tol), info);
        P->state_clobbered = true;                           // until the next segment starts
        if (rc < 0) return rc;
        if (rc == ACS_SOLVED && info[4] <= tol) break;       // polished to tol: st = ACS_SOLVED
        // resume: the scaling, the multiplier and the iterate's x, z back (a
        // polished point that was better but not good enough replaced w, x, z;
        // a rescaling at the next iteration reads x and z), so that the
        // iteration continues as if uninterrupted
        if (cudaMemcpyAsync(P->X.O, P->psaveO, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(P->X.w, P->psaveW, sizeof(double) * P->m, cudaMemcpyDeviceToDevice, P->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(P->x, P->psaveX, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream) != cudaSuccess ||
            cudaMemcpyAsync(P->z, P->psaveZ, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream) != cudaSuccess)
            return ACS_ERR_CUDA;
        P->warm = true;
        P->warm_l = seg.l;
        P->warm_ds = seg.ds;
        P->warm_snorm = seg.snorm;
        P->warm_eta = seg.eta;
        level *= 0.1;
    }
    // the whole solve's counters in the device record (acs_get, the debug getters)
    acs::Control fin;
    if (cudaMemcpy(&fin, P->ctl, sizeof(fin), cudaMemcpyDeviceToHost) != cudaSuccess) return ACS_ERR_CUDA;
    fin.cg_iters = acc.cg_iters;
    fin.n_cg_A = acc.n_cg_A; fin.n_cg_AT = acc.n_cg_AT; fin.n_64_A = acc.n_64_A; fin.n_64_AT = acc.n_64_AT;
    fin.n_cond = acc.n_cond; fin.n_checks = acc.n_checks;
    fin.n_dense_solve = acc.n_dense_solve; fin.n_dense_factor = acc.n_dense_factor;
    fin.n_32_A = acc.n_32_A; fin.n_32_AT = acc.n_32_AT;
    for (int i = 0; i < acs::PH_COUNT; ++i) {
        fin.phase_ns[i] = acc.phase_ns[i];
        fin.phase_n[i] = acc.phase_n[i];
    }
    if (cudaMemcpy(P->ctl, &fin, sizeof(fin), cudaMemcpyHostToDevice) != cudaSuccess) return ACS_ERR_CUDA;
    return st;
}

}  // namespace

extern "C" {

int acs_settings_default(acs_settings* s) {
    if (!s) return ACS_ERR_ARG;
    memset(s, 0, sizeof(*s));
    s->mu = 1.0;
    s->t = 9.2;
    s->cond_first = 300;
    s->cond_period = 100;
    s->cond_list = nullptr;
    s->n_cond_list = 0;
    s->check_every = 10;
    s->precision = ACS_PREC_MIXED;
    s->cg_eta = 0.3;
    s->cg_tol = 1e-12;
    s->cg_max_iter = 500;
    s->cg_refine = 1;
    s->cuda_stream = nullptr;
    s->device = 0;
    s->projection = ACS_PROJ_AUTO;
    s->dense_max_m = 512;
    s->dense_switch_max_m = 1024;
    s->dense_switch_cg = 40;
    s->a_storage = ACS_STORE_FP32;
    s->extrapolation = 0.0;
    s->col_block = -1;
    s->outer32_tol = 1e-5;
    s->splitting = ACS_SPLIT_DR;
    s->polish_tol = 0.0;
    return ACS_SOLVED;
}

const char* acs_status_string(int st) {
    switch (st) {
        case ACS_SOLVED: return "solved";
        case ACS_MAX_ITER: return "iteration limit reached";
        case ACS_POLISH_KEPT: return "polish not better: iterate kept";
        case ACS_ERR_ARG: return "invalid argument";
        case ACS_ERR_CSR: return "malformed CSR matrix";
        case ACS_ERR_CONES: return "invalid cone sizes";
        case ACS_ERR_OOM: return "device out of memory";
        case ACS_ERR_FACTOR: return "projection operator not positive definite";
        case ACS_ERR_DEVICE_TIMEOUT: return "device barrier timed out";
        case ACS_ERR_NUMERICAL: return "non-finite iterate or residual";
        case ACS_ERR_CUDA: return "CUDA runtime error";
        case ACS_ERR_LIMIT: return "size exceeds the entry point's limit";
        default: return "unknown status";
    }
}

const char* acs_version(void) { return kVersion; }

int acs_problem_create(int32_t m, int32_t n, const int64_t* row_ptr, const int32_t* col,
                       const double* val, const double* b, const double* c,
                       int32_t n_orthant, int32_t n_soc, const int32_t* soc_dims,
                       const acs_settings* settings, acs_problem** out) {
    if (!out) return ACS_ERR_ARG;
    *out = nullptr;
    if (m <= 0 || n <= 0 || !row_ptr || !b || !c) return ACS_ERR_ARG;
    acs_settings set;
    if (settings) set = *settings; else acs_settings_default(&set);
    if (!acs::host::valid_settings(set)) return ACS_ERR_ARG;
    // ACS_TRACE_CREATE set: the host time of each step on stderr
    const bool trace = getenv("ACS_TRACE_CREATE") != nullptr;
    auto t_last = std::chrono::steady_clock::now();
    auto step = [&](const char* what) {
        if (!trace) return;
        const auto t = std::chrono::steady_clock::now();
        fprintf(stderr, "acs create: %-10s %8.2f ms\n", what,
                std::chrono::duration<double, std::milli>(t - t_last).count());
        t_last = t;
    };
    const int vrc = acs::host::no_throw(
        [&] { return acs::host::validate(m, n, row_ptr, col, val, b, c, n_orthant, n_soc, soc_dims); });
    step("validate");
    if (vrc != ACS_SOLVED) return vrc;
    if (set.polish_tol > 0 && n_soc > 0) return ACS_ERR_ARG;     // the polish is for LPs
    const int nnz = (int)row_ptr[m];
    Problem* P = new (std::nothrow) Problem();
    if (!P) return ACS_ERR_OOM;
    P->m = m; P->n = n; P->nnz = nnz; P->n_orth = n_orthant; P->n_soc = n_soc;
    P->set = set;
    P->device = set.device;
    if (set.n_cond_list > 0) P->cond_list_host.assign(set.cond_list, set.cond_list + set.n_cond_list);
    P->set.cond_list = nullptr;
    if (cudaSetDevice(P->device) != cudaSuccess) { delete P; return ACS_ERR_CUDA; }
    if (set.cuda_stream) {
        P->stream = (cudaStream_t)set.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking) != cudaSuccess) { delete P; return ACS_ERR_CUDA; }
        P->own_stream = true;
    }
    int rc = ACS_SOLVED;
    if (acs::occupancy_grid(P) != ACS_SOLVED) { free_all(P); delete P; return ACS_ERR_CUDA; }
    step("stream");
    const long long warps = (long long)P->grid32 * acs::kThreads / 32;
    acs::host::HostProblem H;
    acs::host::HostTranspose HT_csr;
    P->full_rows = (long long)nnz == (long long)m * (long long)n;
    P->dense = acs::host::dense_mode(set, m, P->full_rows);
    const bool cb = cb_wanted(set, P->dense);
    // without the column-blocked layout the images are built on the device
    // (the host does the relabelling and the O(m + n) slice tables); a column
    // too long for the device sort falls back to the host builder
    bool on_device = false;
    if (!cb) {
        const int mrc = acs::host::no_throw([&] {
            acs::host::build_meta(m, n, row_ptr, b, c, n_orthant, n_soc, soc_dims, H);
            return ACS_SOLVED;
        });
        if (mrc != ACS_SOLVED) { free_all(P); delete P; return mrc; }
        step("relabel");
        const int gA = acs::host::choose_g(m, nnz, warps), gAT = acs::host::choose_g(n, nnz, warps);
        acs::DeviceSell D;
        int drc = ACS_ERR_OOM;
        try {
            drc = acs::device_sell(P, row_ptr, col, val, H.perm, gA, gAT, D);
        } catch (...) {
            drc = ACS_ERR_OOM;
        }
        step("device build");
        if (drc == ACS_SOLVED) {
            if (adopt_device_sell(P, m, gA, D.sptrA, D.slenA, D.colA, D.valA, D.totA, P->A) ||
                adopt_device_sell(P, n, gAT, D.sptrT, D.slenT, D.colT, D.valT, D.totT, P->AT)) {
                free_all(P); delete P; return ACS_ERR_OOM;
            }
            P->padded_A = D.totA;
            P->padded_AT = D.totT;
            on_device = true;
        } else if (drc != 1) {
            free_all(P); delete P; return drc;
        }
        step("narrow copies");
    }
    if (!on_device) {
        const int brc = acs::host::no_throw([&] {
            return acs::host::build(m, n, row_ptr, col, val, b, c, n_orthant, n_soc, soc_dims, warps, warps, H,
                                    cb ? &HT_csr : nullptr);
        });
        if (brc != ACS_SOLVED) { free_all(P); delete P; return brc; }
        step("build");
    }
    // column-blocked images of A (rows relabelled as above) and A'
    acs::host::HostCb CA, CT;
    bool cb_ok = false;
    if (cb) {
        const int lim = set.col_block > 0 ? std::min(set.col_block, acs::kCbMaxWidth) : acs::kCbMaxWidth;
        const int crc = acs::host::no_throw([&] {
            const int T = acs::host::host_threads(nnz);
            std::vector<long long> beg(m), end(m);
            for (int r = 0; r < m; ++r) { beg[r] = row_ptr[H.perm[r]]; end[r] = row_ptr[H.perm[r] + 1]; }
            if (!acs::host::build_cbsell(m, n, acs::host::cb_width(n, lim), beg, end, col, val, P->grid32, T, CA))
                return ACS_ERR_CSR;
            std::vector<long long> begT(HT_csr.rp.begin(), HT_csr.rp.end() - 1), endT(HT_csr.rp.begin() + 1,
                                                                                     HT_csr.rp.end());
            if (!acs::host::build_cbsell(n, m, acs::host::cb_width(m, lim), begT, endT, HT_csr.rows.data(),
                                         HT_csr.vals.data(), P->grid32, T, CT))
                return ACS_ERR_CSR;
            return ACS_SOLVED;
        });
        cb_ok = crc == ACS_SOLVED;
        HT_csr = acs::host::HostTranspose();
    }
    P->perm = H.perm;
    if (!on_device) {
        P->padded_A = (long long)H.A.col.size();
        P->padded_AT = (long long)H.AT.col.size();
    }
    P->bnorm = H.bnorm;
    P->cnorm = H.cnorm;
    const HostSell& HA = H.A;
    const HostSell& HT = H.AT;
    const std::vector<double>& bperm = H.bperm;
    const std::vector<int>& off = H.soc_off;

    if (!on_device && (acs::host::no_throw([&] { return upload_sell(P, HA, P->A, !cb_ok); }) ||
                       acs::host::no_throw([&] { return upload_sell(P, HT, P->AT, !cb_ok); }))) {
        free_all(P); delete P; return ACS_ERR_OOM;
    }
    step("upload A");
    if (cb_ok) {
        if (acs::host::no_throw([&] { return upload_cb(P, CA, P->Acb); }) ||
            acs::host::no_throw([&] { return upload_cb(P, CT, P->ATcb); })) {
            free_all(P); delete P; return ACS_ERR_OOM;
        }
        P->padded_Acb = (long long)CA.col.size();
        P->padded_ATcb = (long long)CT.col.size();
        // one block of the vector in a pass; in a combine, two tiles of up to
        // kCbCombineMaxGroup blocks
        const int g = std::min(std::max(CA.nblocks, CT.nblocks), acs::kCbCombineMaxGroup);
        P->cb_smem = std::max((int)sizeof(float) * std::max(CA.width, CT.width), 2 * g * acs::kCbWindow * 6);
        P->cb_smem = std::min(P->cb_smem, acs::cb_smem_limit());
        CA = acs::host::HostCb();
        CT = acs::host::HostCb();
    }
    rc |= dalloc(P, &P->soc_off, n_soc + 1);
    rc |= dalloc(P, &P->b, m); rc |= dalloc(P, &P->c, n);
    rc |= dalloc(P, &P->x, n); rc |= dalloc(P, &P->z, n);
    rc |= dalloc(P, &P->ocone, (size_t)n_orthant + n_soc);
    if (!P->cond_list_host.empty()) rc |= dalloc(P, &P->cond_list, P->cond_list_host.size());
    if (rc) { free_all(P); delete P; return ACS_ERR_OOM; }
    if (alloc_outer(P, P->X) || alloc_inner(P, P->V32) || alloc_inner(P, P->V64)) {
        free_all(P); delete P; return ACS_ERR_OOM;
    }
    if (P->dense && (dalloc(P, &P->dM, (size_t)m * m) || dalloc(P, &P->dX, (size_t)m * m))) {
        free_all(P); delete P; return ACS_ERR_OOM;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->device);
    P->max_ctas = (nsm > 0 ? nsm : 1) * 8;
    if (dalloc(P, &P->partials, (size_t)P->max_ctas * acs::kMaxRed) || dalloc(P, &P->flags, P->max_ctas) ||
        dalloc(P, &P->release, 32) || dalloc(P, &P->bcast, acs::kMaxRed) ||
        dalloc(P, &P->ctl, 1)) { free_all(P); delete P; return ACS_ERR_OOM; }
    if (cudaMallocHost(&P->ctl_host, sizeof(acs::Control)) != cudaSuccess) { free_all(P); delete P; return ACS_ERR_OOM; }
    if (cudaEventCreate(&P->ev_launch[0]) != cudaSuccess || cudaEventCreate(&P->ev_launch[1]) != cudaSuccess ||
        cudaEventCreate(&P->ev_polish[0]) != cudaSuccess || cudaEventCreate(&P->ev_polish[1]) != cudaSuccess) {
        free_all(P); delete P; return ACS_ERR_CUDA;
    }
    step("allocate");
    rc = 0;
    rc |= upload(P, P->soc_off, off.data(), n_soc + 1);
    rc |= upload(P, P->b, bperm.data(), m);
    rc |= upload(P, P->c, c, n);
    if (!P->cond_list_host.empty())
        rc |= upload(P, P->cond_list, P->cond_list_host.data(), P->cond_list_host.size());
    rc |= cudaMemsetAsync(P->X.w, 0, sizeof(double) * m, P->stream) != cudaSuccess;
    rc |= cudaMemsetAsync(P->X.q, 0, sizeof(double) * n, P->stream) != cudaSuccess;
    rc |= cudaMemsetAsync(P->ctl, 0, sizeof(acs::Control), P->stream) != cudaSuccess;
    if (rc || cudaStreamSynchronize(P->stream) != cudaSuccess) { free_all(P); delete P; return ACS_ERR_CUDA; }
    if (P->grid32 > P->max_ctas || P->grid64 > P->max_ctas || P->grid32 > 256 || P->grid64 > 256) { free_all(P); delete P; return ACS_ERR_CUDA; }
    step("finish");
    P->create_h2d = P->h2d_bytes;
    P->create_d2h = P->d2h_bytes;
    *out = reinterpret_cast<acs_problem*>(P);
    return ACS_SOLVED;
}

int acs_solve_async(acs_problem* h, double tol, int32_t max_iter) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || !(tol >= 0) || max_iter < 0) return ACS_ERR_ARG;
    P->pol = acs::PolishStats{};
    P->polished_solve = false;
    P->polish_ms = 0.0;
    if (cudaSetDevice(P->device) != cudaSuccess) return ACS_ERR_CUDA;
    return acs::launch_solve(P, tol, max_iter);
}

int acs_solve(acs_problem* h, double tol, int32_t max_iter) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (P && P->set.polish_tol > tol && tol >= 0 && max_iter >= 0) {
        if (cudaSetDevice(P->device) != cudaSuccess) return ACS_ERR_CUDA;
        const int rc = solve_polished(P, tol, max_iter);
        if (rc < 0) return rc;
        return acs_get(h, nullptr, nullptr, nullptr, nullptr, nullptr);
    }
    int rc = acs_solve_async(h, tol, max_iter);
    if (rc != ACS_SOLVED) return rc;
    return acs_get(h, nullptr, nullptr, nullptr, nullptr, nullptr);
}

int acs_get(acs_problem* h, double* x, double* y, double* s, int32_t* iters, double* residuals) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P) return ACS_ERR_ARG;
    if (cudaSetDevice(P->device) != cudaSuccess) return ACS_ERR_CUDA;
    cudaStream_t st = P->stream;
    if (cudaMemcpyAsync(P->ctl_host, P->ctl, sizeof(acs::Control), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ACS_ERR_CUDA;
    if (x && cudaMemcpyAsync(x, P->x, sizeof(double) * P->n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ACS_ERR_CUDA;
    if (s && cudaMemcpyAsync(s, P->z, sizeof(double) * P->n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ACS_ERR_CUDA;
    std::vector<double> wtmp;
    if (y) {
        wtmp.resize(P->m);
        if (cudaMemcpyAsync(wtmp.data(), P->X.w, sizeof(double) * P->m, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return ACS_ERR_CUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return ACS_ERR_CUDA;
    const acs::Control& C = *P->ctl_host;
    if (y)
        for (int r = 0; r < P->m; ++r) y[P->perm[r]] = wtmp[r] / P->set.mu;
    if (iters) *iters = C.l;
    if (residuals) {
        for (int i = 0; i < 6; ++i) residuals[i] = C.res[i];
        residuals[6] = (double)C.cg_iters;
        residuals[7] = (double)C.switched_at;
    }
    int st_code = C.status;
    if (st_code == acs::ST_RUNNING || st_code == acs::ST_SWITCH) st_code = ACS_ERR_CUDA;
    P->last_status = st_code;
    return st_code;
}

// pass counters for the benchmark's byte model.
int acs_debug_counters(acs_problem* h, long long* out6) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || !out6) return ACS_ERR_ARG;
    acs::Control C;
    if (cudaMemcpy(&C, P->ctl, sizeof(C), cudaMemcpyDeviceToHost) != cudaSuccess) return ACS_ERR_CUDA;
    out6[0] = C.n_cg_A; out6[1] = C.n_cg_AT; out6[2] = C.n_64_A; out6[3] = C.n_64_AT;
    out6[4] = C.n_cond; out6[5] = C.n_checks;
    return ACS_SOLVED;
}

int acs_debug_phase_times(acs_problem* h, double* ms, long long* count, int32_t n) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || !ms || !count || n < acs::PH_COUNT) return ACS_ERR_ARG;
    acs::Control C;
    if (cudaStreamSynchronize(P->stream) != cudaSuccess ||
        cudaMemcpy(&C, P->ctl, sizeof(C), cudaMemcpyDeviceToHost) != cudaSuccess)
        return ACS_ERR_CUDA;
    for (int i = 0; i < acs::PH_COUNT; ++i) {
        ms[i] = (double)C.phase_ns[i] * 1e-6;
        count[i] = (long long)C.phase_n[i];
    }
    return acs::PH_COUNT;
}

int acs_debug_barrier_ns(acs_problem* h, int32_t n, double* ns) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || !ns || n <= 0) return ACS_ERR_ARG;
    if (cudaSetDevice(P->device) != cudaSuccess) return ACS_ERR_CUDA;
    return acs::barrier_probe(P, n, ns);
}

int acs_debug_barrier_timeout(acs_problem* h, double* waited_ms) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || !waited_ms) return ACS_ERR_ARG;
    if (cudaSetDevice(P->device) != cudaSuccess) return ACS_ERR_CUDA;
    double ns = 0.0;
    const int rc = acs::barrier_probe(P, 1, &ns, P->grid32 - 1);
    *waited_ms = ns * 1e-6;
    return rc;
}

int acs_debug_sell(int32_t m, int32_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                   int32_t which, int64_t warps, int32_t* info, int32_t* perm, int32_t* sptr, int32_t* slen,
                   int32_t* out_col, double* out_val) {
    if (!info || (which != 0 && which != 1) || warps <= 0 || m <= 0 || n <= 0) return ACS_ERR_ARG;
    return acs::host::no_throw([&]() -> int {
        std::vector<double> b((size_t)m, 0.0), c((size_t)n, 0.0);
        const int v = acs::host::validate(m, n, row_ptr, col, val, b.data(), c.data(), n, 0, nullptr);
        if (v != ACS_SOLVED) return v;
        acs::host::HostProblem H;
        if (acs::host::build(m, n, row_ptr, col, val, b.data(), c.data(), n, 0, nullptr, warps, warps, H) != ACS_SOLVED)
            return ACS_ERR_CSR;
        const acs::host::HostSell& S = which == 0 ? H.A : H.AT;
        info[0] = S.nrows;
        info[1] = S.nslices;
        info[2] = S.g;
        info[3] = (int32_t)S.col.size();
        if (perm) std::copy(H.perm.begin(), H.perm.end(), perm);
        if (sptr) std::copy(S.sptr.begin(), S.sptr.end(), sptr);
        if (slen) std::copy(S.slen.begin(), S.slen.end(), slen);
        if (out_col) std::copy(S.col.begin(), S.col.end(), out_col);
        if (out_val) std::copy(S.val.begin(), S.val.end(), out_val);
        return ACS_SOLVED;
    });
}

int acs_debug_images(acs_problem* h, int32_t which, int32_t* info, int32_t* sptr, int32_t* slen, int32_t* out_col,
                     double* out_val, float* out_v32) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || !info || (which != 0 && which != 1)) return ACS_ERR_ARG;
    const acs::SellMat& M = which == 0 ? P->A : P->AT;
    const long long tot = which == 0 ? P->padded_A : P->padded_AT;
    info[0] = M.nrows; info[1] = M.nslices; info[2] = M.g; info[3] = (int32_t)tot;
    if (cudaSetDevice(P->device) != cudaSuccess || cudaStreamSynchronize(P->stream) != cudaSuccess)
        return ACS_ERR_CUDA;
    if ((sptr && cudaMemcpy(sptr, M.sptr, sizeof(int) * (M.nslices + 1), cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (slen && cudaMemcpy(slen, M.slen, sizeof(int) * M.nslices, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (out_col && cudaMemcpy(out_col, M.col, sizeof(int) * tot, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (out_val && cudaMemcpy(out_val, M.v64, sizeof(double) * tot, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (out_v32 && M.v32 && cudaMemcpy(out_v32, M.v32, sizeof(float) * tot, cudaMemcpyDeviceToHost) != cudaSuccess))
        return ACS_ERR_CUDA;
    return ACS_SOLVED;
}

int acs_debug_cbsell(int32_t m, int32_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                     int32_t which, int32_t width_limit, int32_t ctas, int64_t* info, int32_t* perm,
                     int32_t* sptr, uint16_t* rowid, uint16_t* out_col, float* out_val, int32_t* cta_beg,
                     uint32_t* cend, uint16_t* ipos) {
    if (!info || (which != 0 && which != 1) || width_limit < 4 || ctas <= 0 || m <= 0 || n <= 0)
        return ACS_ERR_ARG;
    return acs::host::no_throw([&]() -> int {
        std::vector<double> b((size_t)m, 0.0), c((size_t)n, 0.0);
        const int v = acs::host::validate(m, n, row_ptr, col, val, b.data(), c.data(), n, 0, nullptr);
        if (v != ACS_SOLVED) return v;
        acs::host::HostProblem H;
        acs::host::HostTranspose T;
        if (acs::host::build(m, n, row_ptr, col, val, b.data(), c.data(), n, 0, nullptr, 1, 1, H, &T) !=
            ACS_SOLVED)
            return ACS_ERR_CSR;
        const int lim = std::min(width_limit, acs::kCbMaxWidth);
        const int th = acs::host::host_threads(row_ptr[m]);
        acs::host::HostCb C;
        bool ok;
        if (which == 0) {
            std::vector<long long> beg(m), end(m);
            for (int r = 0; r < m; ++r) { beg[r] = row_ptr[H.perm[r]]; end[r] = row_ptr[H.perm[r] + 1]; }
            ok = acs::host::build_cbsell(m, n, acs::host::cb_width(n, lim), beg, end, col, val, ctas, th, C);
        } else {
            std::vector<long long> beg(T.rp.begin(), T.rp.end() - 1), end(T.rp.begin() + 1, T.rp.end());
            ok = acs::host::build_cbsell(n, m, acs::host::cb_width(m, lim), beg, end, T.rows.data(), T.vals.data(),
                                         ctas, th, C);
        }
        if (!ok) return ACS_ERR_CSR;
        info[0] = C.nrows; info[1] = C.ncols; info[2] = C.width; info[3] = C.nblocks; info[4] = C.nsl;
        info[5] = (int64_t)C.col.size();
        if (perm) std::copy(H.perm.begin(), H.perm.end(), perm);
        if (sptr) std::copy(C.sptr.begin(), C.sptr.end(), sptr);
        if (rowid) std::copy(C.rowid.begin(), C.rowid.end(), rowid);
        if (out_col) std::copy(C.col.begin(), C.col.end(), out_col);
        if (out_val) std::copy(C.val.begin(), C.val.end(), out_val);
        if (cta_beg) std::copy(C.cta_beg.begin(), C.cta_beg.end(), cta_beg);
        if (cend) std::copy(C.cend.begin(), C.cend.end(), cend);
        if (ipos) std::copy(C.ipos.begin(), C.ipos.end(), ipos);
        return ACS_SOLVED;
    });
}

int acs_debug_pass_counts(acs_problem* h, int64_t* out, int32_t n) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || !out || n < 12) return ACS_ERR_ARG;
    if (cudaSetDevice(P->device) != cudaSuccess) return ACS_ERR_CUDA;
    acs::Control C;
    if (cudaStreamSynchronize(P->stream) != cudaSuccess ||
        cudaMemcpy(&C, P->ctl, sizeof(C), cudaMemcpyDeviceToHost) != cudaSuccess)
        return ACS_ERR_CUDA;
    out[0] = C.n_cg_A; out[1] = C.n_cg_AT; out[2] = C.n_64_A; out[3] = C.n_64_AT;
    out[4] = C.n_cond; out[5] = C.n_checks; out[6] = C.n_32_A; out[7] = C.n_32_AT;
    out[8] = C.outer32_end; out[9] = C.l; out[10] = C.cg_iters; out[11] = C.switched_at;
    if (n < 16) return 12;
    out[12] = P->pol.attempts; out[13] = P->pol.taken; out[14] = P->pol.corrections; out[15] = P->pol.factored;
    if (n < 18) return 16;
    out[16] = P->pol.support; out[17] = P->pol.support_entries;
    return 18;
}

int acs_bench_passes(acs_problem* h, int32_t kind, int32_t reps, int32_t smem_bytes, double* us_per_rep) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || !us_per_rep || kind < 0 || kind > 21) return ACS_ERR_ARG;
    if (cudaSetDevice(P->device) != cudaSuccess) return ACS_ERR_CUDA;
    return acs::pass_bench(P, kind, reps, smem_bytes < 0 ? P->cb_smem : smem_bytes, us_per_rep);
}

int acs_debug_layout(acs_problem* h, int64_t* out, int32_t n) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || !out || n < 10) return ACS_ERR_ARG;
    out[0] = P->Acb.nblocks > 0 ? 1 : 0;
    out[1] = P->Acb.nblocks; out[2] = P->Acb.width; out[3] = P->padded_Acb;
    out[4] = P->ATcb.nblocks; out[5] = P->ATcb.width; out[6] = P->padded_ATcb;
    out[7] = P->cb_smem; out[8] = P->padded_A; out[9] = P->padded_AT;
    if (n < 12) return 10;
    out[10] = P->A.nslices; out[11] = P->AT.nslices;
    if (n < 14) return 12;
    out[12] = P->create_h2d; out[13] = P->create_d2h;
    return 14;
}

int acs_debug_to_bf16(int64_t n, const double* v, uint16_t* out) {
    if (n < 0 || (n > 0 && (!v || !out))) return ACS_ERR_ARG;
    for (int64_t k = 0; k < n; ++k) out[k] = acs::host::to_bf16(v[k]);
    return ACS_SOLVED;
}

int acs_last_launch_ms(acs_problem* h, double* ms) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || !ms) return ACS_ERR_ARG;
    if (P->polished_solve) {
        *ms = P->seg_ms;
        return ACS_SOLVED;
    }
    float f = 0.f;
    if (cudaEventSynchronize(P->ev_launch[1]) != cudaSuccess ||
        cudaEventElapsedTime(&f, P->ev_launch[0], P->ev_launch[1]) != cudaSuccess)
        return ACS_ERR_CUDA;
    *ms = (double)f;
    return ACS_SOLVED;
}

int acs_last_polish_ms(acs_problem* h, double* ms) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || !ms) return ACS_ERR_ARG;
    *ms = P->polish_ms;
    return ACS_SOLVED;
}

int acs_problem_info(acs_problem* h, int32_t* out8) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || !out8) return ACS_ERR_ARG;
    out8[0] = P->m; out8[1] = P->n; out8[2] = P->nnz;
    out8[3] = (int32_t)std::min<long long>(P->padded_A, INT32_MAX);
    out8[4] = (int32_t)std::min<long long>(P->padded_AT, INT32_MAX);
    out8[5] = P->grid32; out8[6] = P->grid64; out8[7] = acs::kThreads;
    return ACS_SOLVED;
}

int acs_polish(acs_problem* h, int32_t rounds, double* info) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || rounds < 1 || rounds > 8 || P->n_soc > 0 || P->solves == 0) return ACS_ERR_ARG;
    const int st = acs_get(h, nullptr, nullptr, nullptr, nullptr, nullptr);   // waits for the solve
    if (st < 0) return st == ACS_ERR_CUDA ? st : ACS_ERR_ARG;
    double local[7];
    const int rc = polish_once(P, rounds, 1e-13, info ? info : local);
    if (rc < 0) return rc;
    P->state_clobbered = true;
    return rc;
}

int acs_get_state(acs_problem* h, double* s_dr, double* O, double* w, int32_t* l, double* step) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || P->state_clobbered) return ACS_ERR_ARG;
    if (cudaSetDevice(P->device) != cudaSuccess) return ACS_ERR_CUDA;
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) return ACS_ERR_CUDA;
    acs::Control C;
    if (cudaMemcpy(&C, P->ctl, sizeof(C), cudaMemcpyDeviceToHost) != cudaSuccess) return ACS_ERR_CUDA;
    if (s_dr && cudaMemcpy(s_dr, P->X.s, sizeof(double) * P->n, cudaMemcpyDeviceToHost) != cudaSuccess) return ACS_ERR_CUDA;
    if (O && cudaMemcpy(O, P->X.O, sizeof(double) * P->n, cudaMemcpyDeviceToHost) != cudaSuccess) return ACS_ERR_CUDA;
    if (w) {
        std::vector<double> t(P->m);
        if (cudaMemcpy(t.data(), P->X.w, sizeof(double) * P->m, cudaMemcpyDeviceToHost) != cudaSuccess) return ACS_ERR_CUDA;
        for (int r = 0; r < P->m; ++r) w[P->perm[r]] = t[r];
    }
    if (l) *l = C.l;
    if (step) { step[0] = C.ds; step[1] = C.snorm; step[2] = C.eta; }
    return ACS_SOLVED;
}

int acs_set_state(acs_problem* h, const double* s_dr, const double* O, const double* w, int32_t l,
                  const double* step) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P || !s_dr || !O || !w || l < 0) return ACS_ERR_ARG;
    if (!finite_all(s_dr, P->n) || !finite_all(O, P->n) || !finite_all(w, P->m)) return ACS_ERR_ARG;
    for (int j = 0; j < P->n; ++j)
        if (!(O[j] > 0)) return ACS_ERR_ARG;
    if (cudaSetDevice(P->device) != cudaSuccess) return ACS_ERR_CUDA;
    int rc = 0;
    std::vector<double> wp(P->m);
    for (int r = 0; r < P->m; ++r) wp[r] = w[P->perm[r]];
    rc |= upload(P, P->X.s, s_dr, P->n);
    rc |= upload(P, P->X.w, wp.data(), P->m);
    rc |= upload(P, P->X.O, O, P->n);
    if (rc || cudaStreamSynchronize(P->stream) != cudaSuccess) return ACS_ERR_CUDA;
    P->warm = true;
    P->warm_l = l;
    P->warm_ds = step ? step[0] : INFINITY;
    P->warm_snorm = step ? step[1] : 0.0;
    P->warm_eta = (step && step[2] > 0) ? step[2] : P->set.cg_eta;
    return ACS_SOLVED;
}

void acs_problem_destroy(acs_problem* h) {
    Problem* P = reinterpret_cast<Problem*>(h);
    if (!P) return;
    cudaSetDevice(P->device);
    if (P->stream) cudaStreamSynchronize(P->stream);
    free_all(P);
    delete P;
}

}  // extern "C"
