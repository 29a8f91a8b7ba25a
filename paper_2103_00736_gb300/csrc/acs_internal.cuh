// Internal types of the GB300 conic solver: device buffers of one problem,
// the per-launch parameter block of the persistent iteration kernel, and the
// device-side control block.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <utility>
#include <vector>

#include "../../include/acs.h"

namespace acs {

constexpr int kThreads = 1024;          // threads per CTA of the persistent kernel
constexpr int kWarps = kThreads / 32;
constexpr int kMaxRed = 8;              // doubles reduced per grid reduction
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // 2 s per barrier
// FP32 outer passes end after this many KKT checks without a 10 % fall of the
// largest residual (they have reached the rounding floor of FP32 products)
constexpr int kOuter32FlatChecks = 10;

// device-side status value of a solve still in progress
enum : int {
    ST_RUNNING = 100,
    ST_SWITCH = 101,   // FP32 correction solve handed over to FP64
    ST_PAUSED = 102    // a time-sliced solve stopped at its deadline; resumable
};

// phases of the persistent kernel, for the per-phase time record
enum Phase : int {
    PH_COND_O = 0, PH_COND_APPLY, PH_BTILDE, PH_QREFRESH, PH_ABS, PH_RHS, PH_CG_AT, PH_CG_A,
    PH_CG_VEC, PH_UPDATE, PH_KKT, PH_DENSE_FACTOR, PH_DENSE_SOLVE,
    PH_CG_TCOMB,     // column-blocked CG: t = O^2 (A'u) from the partial sums, and u'Mu
    PH_RHS_COMB,     // FP32 outer passes: the projection residual from the partial sums
    PH_UPD_COMB,     // FP32 outer passes: q = A_hat' w from the partial sums and the update
    PH_DENSE_ASSEMBLE,   // cached operator: M = A O^2 A' (PH_DENSE_FACTOR: its Cholesky steps)
    PH_DENSE_INVERSE,    // cached operator: L^{-1}
    PH_COUNT
};

// Control block: lives in device memory for the whole solve; the host reads
// it back at acs_get.  Written only by CTA 0 at the end of a launch.
struct Control {
    int status;           // ST_RUNNING, ACS_SOLVED, ACS_MAX_ITER or an error
    int err;              // first device-side error (0 = none); checked at every barrier
    int l;                // iterations completed
    int pad0;
    long long cg_iters;   // conjugate-gradient iterations, all outer iterations
    int switched_at;      // iteration at which the FP32 correction solve handed over (0 = never)
    int pad1;
    double res[6];        // r_p, r_d, r_gap, r_cone, obj_p, obj_d at the last check
    double ds;            // ||s_l - s_{l-1}|| of the last iteration
    double snorm;         // ||s_l||
    double eta;           // current inexactness factor of the projection solve
    // pass counters (for the algorithmic-byte model of the benchmark)
    long long n_cg_A, n_cg_AT, n_64_A, n_64_AT, n_cond, n_checks;
    long long n_dense_solve, n_dense_factor;   // cached-operator corrections and factorisations
    long long n_32_A, n_32_AT;                 // FP32 outer passes (projection residual, update)
    int outer32_end;      // iteration at which the FP32 outer passes ended (0 = not yet)
    int pad2;
    int stage;            // loop that runs the solve: 0 = FP32 correction CG, 1 = FP64 loop
    int dense_on;         // the cached dense operator is in use (kept across pauses)
    int dense_failed;     // its factorisation failed for this solve
    int win_it;           // outer iterations since the last rescaling
    long long win_cg;     // CG iterations since the last rescaling (switch to the cached operator)
    int extrap_ok;        // wp, qp hold the previous iteration's w, q in the current scaling
    int factor_ok;        // the problem's own cached factor is that of the current O
    unsigned bar_count, bar_gen;
    unsigned long long bar_count64;   // monotonic barrier arrival counter of the current solve
    // nanoseconds spent in each phase (from one barrier exit to the next, as
    // seen by CTA 0), accumulated over the solve, and the number of phases run
    unsigned long long phase_ns[PH_COUNT];
    unsigned long long phase_n[PH_COUNT];
};

// Outer iteration state, always FP64 (Algorithm 2 in the scaled space).
struct Outer {
    double *s, *p, *g, *q, *w, *chat, *btil, *O;
    double *wp, *qp;      // w and q = A_hat' w of the previous iteration (extrapolated start)
};
// Inner projection-solve (CG) state in precision T (Chronopoulos-Gear CG:
// r residual, u = J^{-1} r, p direction, sv = M p, au = M u, t = O^2 A' u).
template <typename T>
struct Inner {
    T *r, *u, *p, *sv, *au, *t, *jinv, *O2;
};

// Sliced ELLPACK, one warp per slice, G lanes per row (G in 1..32, a power
// of two): slice sl holds rows sl*(32/G) ... + 32/G - 1; entry k of local row
// r sits at sptr[sl] + 32*(k/G) + r*G + k%G, so every chunk of 32 entries is
// contiguous.  Rows shorter than G*slen[sl] are padded with (col 0, val 0).
struct SellMat {
    int nrows, nslices, g;
    const int* sptr;       // [nslices + 1] start of each slice
    const int* slen;       // [nslices] 32-entry chunks in the slice
    const int* col;        // [sptr[nslices]]
    const float* v32;
    const double* v64;
    const unsigned short* v16;   // BF16 bit patterns of the values (BF16 storage of A), else NULL
};

// Column-blocked sliced ELLPACK of the FP32 passes of the single-problem
// launch (layout and host builder in acs_cbsell.cuh); nblocks = 0: not used.
// Lane r of item (block b, slice q) holds row
// (q / kCbSliceWin) * kCbWindow + rowid[item * 32 + r] (kCbNoRow: none).
constexpr int kCbWindow = 2048;                 // rows sorted together by their count in a block
constexpr int kCbSliceWin = kCbWindow / 32;     // slices per window
constexpr unsigned short kCbNoRow = 0xFFFF;
constexpr int kCbCombineMaxGroup = 7;           // blocks per tile of a combine phase
struct CbMat {
    int nrows, ncols, width, nblocks, nsl;      // nsl = slices per block = ceil(nrows / 32)
    int ctas;                                   // CTAs the item ranges were dealt to
    const int* sptr;                            // [nblocks * nsl + 1]
    const unsigned short* rowid;                // [nblocks * nsl * 32]
    const unsigned short* col;                  // [sptr[last]]
    const float* val;                           // [sptr[last]]
    const int* cta_beg;                         // [ctas + 1]
    const unsigned* cend;                       // item-end marks, one bit per chunk of 32 entries
    const unsigned short* ipos;                 // [nblocks * nsl * 32] slot of each row in its window
    float* part;                                // [nblocks * nsl * 32] partial sums of the last pass,
                                                //   in slot order (item * 32 + lane)
};

// Everything one launch of the iteration kernel needs (passed by value).
template <typename T>
struct IterParams {
    int m, n, n_orth, n_soc;
    SellMat A, AT;                                    // A (rows relabelled) and A'
    const int* soc_off;                               // n_soc + 1 absolute offsets
    const double* b; const double* c;
    double bnorm, cnorm;
    Outer X;
    Inner<T> V;
    double* x; double* z;                             // FP64 iterates (steps 20-21)
    double* ocone;                                    // log o per cone (orthant coords first)
    double* partials;                                 // [gridDim.x * kMaxRed]
    unsigned* flags;                                  // [gridDim.x] barrier arrival flags
    unsigned* release;                                // barrier release flag
    double* bcast;                                    // [kMaxRed] reduced values
    Control* ctl;
    // settings
    double mu, t_cond;
    int cond_first, cond_period;
    const int* cond_list; int n_cond_list;
    int check_every, max_iter;
    double tol, cg_eta, cg_tol, cg_relfloor;
    int cg_max;
    int refresh;                                      // recompute c_hat, b_tilde, J, q first
    int refine;                                       // correction solves per iteration
    int switch_ok;                                    // FP32 launch may hand over to FP64
    int dense;                                        // cached dense projection operator (FP64 loop):
                                                      // 0 = never, 1 = from the start, 2 = when CG stalls
    long long switch_budget;                          // CG iterations since the last rescaling that switch
    double* dM; double* dX;                           // its scratch: single-problem launch, or a member
                                                      // that keeps its own (NULL: the team's)
    int own_scratch;                                  // dM/dX belong to this problem and outlive a launch
    double extrap;                                    // factor of the extrapolated start of the projection
                                                      // solve (0 = start from the previous w)
    CbMat Acb, ATcb;                                  // column-blocked FP32 images of A and A'
                                                      // (FP32 loop of the single-problem launch only)
    int outer32;                                      // FP32 outer passes (rhs, update) until the
    double outer32_tol;                               //   KKT residuals reach outer32_tol
    int admm;                                         // ADMM form of the splitting (Section III-B)
    int outer32_l2;                                   // FP32 outer products on the L2-gather layout
                                                      // (FP32 loop of a segment ending at a polish level)
    int full_rows;                                    // every row of A holds every column (dense
                                                      // workloads): the cached operator's M is
                                                      // assembled by a tiled product
};

struct PolishStats {
    long long attempts = 0, taken = 0, corrections = 0, factored = 0;
    long long support = 0, support_entries = 0;   // |B| and stored entries of A_B of the last polish
};

// Device memory of the single-problem API through a per-device cache of
// released blocks (acs_alloc.cu): *got receives the block's size.
void* dev_alloc(int device, size_t bytes, size_t* got);
void dev_release(int device, void* p, size_t bytes);

struct Problem {
    int m = 0, n = 0, nnz = 0, n_orth = 0, n_soc = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    acs_settings set{};
    std::vector<int> cond_list_host;
    int* cond_list = nullptr;
    double bnorm = 0, cnorm = 0;
    // matrix: A with its rows relabelled by perm (row i of the device matrix
    // is row perm[i] of the caller's A; b, y and w live in that order)
    SellMat A{}, AT{};
    long long padded_A = 0, padded_AT = 0;
    long long padded_Acb = 0, padded_ATcb = 0;   // stored entries of the column-blocked images
    std::vector<int> perm;
    int* soc_off = nullptr;
    double *b = nullptr, *c = nullptr;
    // state
    Outer X{};
    Inner<float> V32{};
    Inner<double> V64{};
    double *x = nullptr, *z = nullptr, *ocone = nullptr;
    double* partials = nullptr;
    unsigned* flags = nullptr;
    unsigned* release = nullptr;
    double* bcast = nullptr;
    int max_ctas = 0;
    Control* ctl = nullptr;
    Control* ctl_host = nullptr;         // pinned mirror
    int grid32 = 0, grid64 = 0;
    bool warm = false;                   // acs_set_state called
    long long solves = 0;                // acs_solve_async calls
    bool state_clobbered = false;        // a polish overwrote the iteration state
    double *px = nullptr, *pw = nullptr, *pz = nullptr, *pwork = nullptr, *pres = nullptr;   // polish (lazy)
    double *pdM = nullptr, *pdX = nullptr;   // polish's factored A_B A_B' when the handle has no scratch
    int *bcol = nullptr, *bsptr = nullptr, *bslen = nullptr, *bcnt = nullptr;   // A_B of the polish (lazy)
    double* bval = nullptr;
    float* bval32 = nullptr;                  // A_B's FP32 values (FP32 polish corrections)
    long long padded_B = 0;
    // bytes copied host -> device and device -> host: running counts of the
    // uploads and of the device build's copies, and their values when
    // acs_problem_create returned
    long long h2d_bytes = 0, d2h_bytes = 0;
    long long create_h2d = 0, create_d2h = 0;
    double* psaveO = nullptr;                 // the scaling O, the multiplier w and the iterate's
    double* psaveW = nullptr;                 //   x, z kept across a polish of a polished solve
    double *psaveX = nullptr, *psaveZ = nullptr;
    PolishStats pol;                          // polish attempts of the last solve (or acs_polish calls)
    int warm_l = 0;
    double warm_ds = INFINITY, warm_snorm = 0.0, warm_eta = 0.3;
    int last_status = ACS_MAX_ITER;
    int dense = 0;                       // cached dense operator: 0 never, 1 always, 2 when CG stalls
    double *dM = nullptr, *dX = nullptr; // its scratch, [m * m] each
    CbMat Acb{}, ATcb{};                 // column-blocked FP32 images (nblocks = 0: not built)
    int cb_smem = 0;                     // dynamic shared memory of the FP32 launch (bytes)
    std::vector<std::pair<void*, size_t>> allocations;   // device blocks owned (address, size)
    // count elements of T from the device cache, owned by the problem
    template <typename T>
    bool alloc(T** out, size_t count) {
        size_t got = 0;
        void* q = dev_alloc(device, (count > 0 ? count : 1) * sizeof(T), &got);
        *out = static_cast<T*>(q);
        if (!q) return false;
        allocations.emplace_back(q, got);
        return true;
    }
    cudaEvent_t ev_launch[2] = {nullptr, nullptr};   // bracket the last persistent launch
    cudaEvent_t ev_polish[2] = {nullptr, nullptr};   // bracket the last polish launch
    double seg_ms = 0.0;                     // a polished solve: its iteration launches' device time
    double polish_ms = 0.0;                  // ... and its polish launches' (or the last acs_polish's)
    bool polished_solve = false;             // the last acs_solve ran with polish_tol
    bool full_rows = false;                  // nnz = m n: every row holds every column
    bool outer_f32 = false;                  // the next launch's FP32 loop uses FP32 outer products
};

// launches (acs_iter.cu)
int launch_solve(Problem* P, double tol, int max_iter);
// Sliced-ELLPACK images of A (rows in the order perm) and A' built on the
// device (acs_devbuild.cu): device col/value arrays (owned by P) and the
// host slice tables.  Returns ACS_SOLVED, 1 if a column is too long for the
// device sort (build on the host instead), or an error.
struct DeviceSell {
    std::vector<int> sptrA, slenA, sptrT, slenT;
    int *colA = nullptr, *colT = nullptr;
    double *valA = nullptr, *valT = nullptr;
    long long totA = 0, totT = 0;
};
int device_sell(Problem* P, const int64_t* row_ptr, const int32_t* col, const double* val,
                const std::vector<int>& perm, int gA, int gAT, DeviceSell& out);
// The crossover polish's A_B (rows of A on the support x > z of the current
// iterate) on the device; sets X.O to the support's indicator.
int support_rows(Problem* P, SellMat& out, bool with_f32);
// LP crossover polish of the current iterate into px, pw, pz; pres[0..5] its
// residuals, pres[8..12] {|B|, CG iterations x, y, 1 = completed, 1 =
// factored}.  rel: the solves stop at rel times their first residual (or at
// its rounding floor).
int launch_polish(Problem* P, int rounds, double rel);
int occupancy_grid(Problem* P);
int cb_smem_limit();
int pass_bench(Problem* P, int kind, int reps, int smem_bytes, double* us);
int barrier_probe(Problem* P, int n, double* ns_per_barrier, int absent = -1);

}  // namespace acs
