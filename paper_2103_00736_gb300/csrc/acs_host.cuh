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
#include <vector>

#include "../../include/acs.h"

namespace acs {
namespace host {

constexpr int kSortWindow = 2048;   // rows of A are sorted by length within windows of this size

inline bool finite_all(const double* v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

constexpr int kDenseLimit = 4096;   // largest m for the cached dense projection operator

// Settings checks shared by every entry point that takes acs_settings.
inline bool valid_settings(const acs_settings& set) {
    return set.mu > 0 && set.t > 0 && set.check_every > 0 && set.cg_max_iter > 0 && set.cg_refine > 0 &&
           set.cg_refine <= 8 && set.cg_tol >= 0 && set.cg_eta >= 0 && set.cond_period >= 0 && set.cond_first >= 0 &&
           set.n_cond_list >= 0 && !(set.n_cond_list > 0 && !set.cond_list) &&
           (set.precision == ACS_PREC_MIXED || set.precision == ACS_PREC_FP64) &&
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
// and at least 8 * dense_switch_cg.
inline long long switch_budget(const acs_settings& set, int m, long long nnz) {
    const double f = 0.3 * (double)m * (double)m * (double)m / (double)(nnz > 0 ? nnz : 1);
    return std::max((long long)8 * set.dense_switch_cg, (long long)f);
}

// How a problem with m constraints applies the projection: 0 = CG only,
// 1 = the cached dense operator from the first iteration, 2 = CG, switching
// to the cached operator if CG stalls.
inline int dense_mode(const acs_settings& set, int m) {
    if (set.projection == ACS_PROJ_DENSE) return m <= kDenseLimit ? 1 : 0;
    if (set.projection != ACS_PROJ_AUTO) return 0;
    if (m <= set.dense_max_m) return 1;
    if (set.dense_switch_cg > 0 && m <= set.dense_switch_max_m) return 2;
    return 0;
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
    for (int i = 0; i < m; ++i) {
        int prev = -1;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            const int j = col[k];
            if (j < 0 || j >= n || j <= prev) return ACS_ERR_CSR;
            prev = j;
        }
    }
    if (!finite_all(val, nnz) || !finite_all(b, m) || !finite_all(c, n)) return ACS_ERR_ARG;
    if (n_orthant < 0 || n_soc < 0 || (n_soc > 0 && !soc_dims)) return ACS_ERR_CONES;
    int64_t tot = n_orthant;
    for (int i = 0; i < n_soc; ++i) {
        if (soc_dims[i] < 2) return ACS_ERR_CONES;
        tot += soc_dims[i];
    }
    if (tot != n) return ACS_ERR_CONES;
    return ACS_SOLVED;
}

// Host image of a sliced-ELLPACK matrix with G lanes per row.
struct HostSell {
    int nrows = 0, nslices = 0, g = 1;
    std::vector<int> sptr, slen, col;
    std::vector<double> val;
};

// Rows are given by (beg[r], end[r]) ranges into (cols, vals); padding
// entries repeat column 0 with value 0.  nslices = -1 if the padded size
// does not fit 32-bit offsets.
inline HostSell build_sell(int nrows, int g, const std::vector<long long>& beg, const std::vector<long long>& end,
                           const int* cols, const double* vals) {
    HostSell H;
    const int h = 32 / g;                     // rows per slice
    H.nrows = nrows;
    H.g = g;
    H.nslices = (nrows + h - 1) / h;
    H.sptr.assign(H.nslices + 1, 0);
    H.slen.assign(H.nslices, 0);
    long long total = 0;
    for (int sl = 0; sl < H.nslices; ++sl) {
        long long mx = 0;
        for (int r = sl * h; r < std::min(nrows, sl * h + h); ++r) mx = std::max(mx, end[r] - beg[r]);
        const long long chunks = (mx + g - 1) / g;
        H.slen[sl] = (int)chunks;
        H.sptr[sl] = (int)std::min<long long>(total, INT32_MAX);
        total += 32 * chunks;
    }
    H.sptr[H.nslices] = (int)std::min<long long>(total, INT32_MAX);
    if (total >= INT32_MAX) { H.col.clear(); H.nslices = -1; return H; }
    H.col.assign(total, 0);
    H.val.assign(total, 0.0);
    for (int sl = 0; sl < H.nslices; ++sl)
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
inline int build(int32_t m, int32_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                 const double* b, const double* c, int32_t n_orthant, int32_t n_soc, const int32_t* soc_dims,
                 long long warps_A, long long warps_AT, HostProblem& H) {
    const int nnz = (int)row_ptr[m];
    // relabel the constraints: sort rows by length (descending) within windows,
    // so that the rows of a slice have similar lengths and padding is small
    std::vector<int>& perm = H.perm;
    perm.resize(m);
    for (int i = 0; i < m; ++i) perm[i] = i;
    for (int w0 = 0; w0 < m; w0 += kSortWindow) {
        const int w1 = std::min(m, w0 + kSortWindow);
        std::stable_sort(perm.begin() + w0, perm.begin() + w1, [&](int a, int b2) {
            return (row_ptr[a + 1] - row_ptr[a]) > (row_ptr[b2 + 1] - row_ptr[b2]);
        });
    }
    {
        std::vector<long long> beg(m), end(m);
        for (int r = 0; r < m; ++r) { beg[r] = row_ptr[perm[r]]; end[r] = row_ptr[perm[r] + 1]; }
        H.A = build_sell(m, choose_g(m, nnz, warps_A), beg, end, col, val);
    }
    {
        // A' by counting sort over the relabelled rows
        std::vector<long long> rpT(n + 1, 0);
        for (int k = 0; k < nnz; ++k) rpT[col[k] + 1]++;
        for (int j = 0; j < n; ++j) rpT[j + 1] += rpT[j];
        std::vector<int> ciT(nnz);
        std::vector<double> valT(nnz);
        std::vector<long long> cur(rpT.begin(), rpT.end() - 1);
        for (int r = 0; r < m; ++r) {
            const int i = perm[r];
            for (long long k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                const long long pos = cur[col[k]]++;
                ciT[pos] = r;
                valT[pos] = val[k];
            }
        }
        std::vector<long long> beg(rpT.begin(), rpT.end() - 1), end(rpT.begin() + 1, rpT.end());
        H.AT = build_sell(n, choose_g(n, nnz, warps_AT), beg, end, ciT.data(), valT.data());
    }
    if (H.A.nslices < 0 || H.AT.nslices < 0) return ACS_ERR_CSR;
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
    return ACS_SOLVED;
}

}  // namespace host
}  // namespace acs
