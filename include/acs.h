/*
 * acs.h -- C ABI of the GB300 adaptive-conditioning conic solver.
 *
 * Solves  min c'x  s.t.  Ax = b,  x in K   (arXiv 2103.00736, Section II, Eq. (1))
 * and its dual  max b'y  s.t.  A'y + z = c,  z in K  (Eq. (2)),
 * where K is a product of Lorentz cones.  The nonnegative orthant is the
 * product of size-1 Lorentz cones; in this ABI its coordinates come first,
 * [0, n_orthant), followed by the cones of size >= 2 in the order given.
 *
 * The method is Algorithm 2 of the paper (Algorithm 1 plus adaptive
 * conditioning, Section IV) run on one GPU: every iteration applies the
 * cone reflection abs_K (Definition 1), the reflection through the range of
 * (A O)' by a Jacobi-preconditioned conjugate-gradient solve with
 * M = (A O)(A O)', the splitting update, and at the iterations of the
 * schedule L the diagonal rescaling O of Algorithm 2, steps 5-14.
 *
 * Conventions
 *  - All pointers passed to acs_problem_create / acs_get / acs_get_state /
 *    acs_set_state are HOST pointers owned by the caller; they are read or
 *    written only during the call.  The library copies the data to the
 *    device and owns every device buffer it allocates until
 *    acs_problem_destroy.
 *  - A handle is not thread-safe: use one handle per host thread, or the
 *    batch API.
 *  - Return codes: 0 = ACS_SOLVED; positive values are terminal statuses
 *    whose results are still valid (ACS_MAX_ITER); negative values are
 *    errors.  No error path traps the GPU: device-side failures (a grid
 *    barrier that times out, a non-finite residual, a failed CG) are
 *    reported through these codes and leave the CUDA context usable.
 */
#ifndef ACS_H
#define ACS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ACS_SOLVED = 0,          /* all relative KKT residuals <= tol                   */
    ACS_MAX_ITER = 1,        /* iteration limit reached; results/residuals valid    */
    ACS_POLISH_KEPT = 2,     /* acs_polish: the polished point was not better; the
                                iterate is kept unchanged                           */
    ACS_ERR_ARG = -1,        /* bad argument (NULL pointer, size <= 0, bad setting) */
    ACS_ERR_CSR = -2,        /* malformed CSR: row_ptr not monotone, col out of
                                range or unsorted/duplicate within a row, empty row */
    ACS_ERR_CONES = -3,      /* cone sizes do not add up to n, or a size < 2        */
    ACS_ERR_OOM = -4,        /* device (or host) allocation failed                  */
    ACS_ERR_FACTOR = -5,     /* M = (AO)(AO)' not positive definite (CG breakdown)  */
    ACS_ERR_DEVICE_TIMEOUT = -6, /* a device-side grid barrier did not complete   */
    ACS_ERR_NUMERICAL = -7,  /* NaN or Inf in the iterates or residuals             */
    ACS_ERR_CUDA = -8,       /* a CUDA runtime call failed                          */
    ACS_ERR_LIMIT = -9       /* a size exceeds a fixed limit of the entry point     */
};

enum { ACS_PREC_MIXED = 0, ACS_PREC_FP32 = 1, ACS_PREC_FP64 = 2 };

typedef struct acs_problem acs_problem;

typedef struct {
    double mu;               /* splitting parameter mu > 0 (Algorithm 1 Require); default 1   */
    double t;                /* conditioning cap t > 0 (Algorithm 2 step 11): the spread
                                max(O)/min(O) is at most e^t; default 9.2 (LP experiments)     */
    int32_t cond_first;      /* schedule L = {cond_first, cond_first + cond_period, ...}
                                plus cond_list; 0 disables the periodic part; l = 1 always
                                conditions (Algorithm 2 step 4); default 300                   */
    int32_t cond_period;     /* default 100                                                    */
    const int32_t* cond_list;/* extra conditioning iterations (host, copied), may be NULL    */
    int32_t n_cond_list;
    int32_t check_every;     /* KKT residual check period in iterations; default 10           */
    int32_t precision;       /* ACS_PREC_MIXED (default): FP64 outer iteration and residuals,
                                projection solve by an FP32 correction CG (mixed-precision
                                refinement), handed over to an FP64 correction CG for the
                                rest of the solve if the FP32 one cannot reach the accuracy
                                the iteration needs; ACS_PREC_FP32: as MIXED, and the two
                                matrix products of the outer iteration (the projection
                                residual b_tilde - A_hat (p + q) and the update's A_hat' w)
                                are FP32 column-blocked passes too until every KKT residual
                                is <= outer32_tol or stops falling, after which they are FP64
                                (the polish that finishes the solve); needs the column-
                                blocked layout (col_block >= 0, FP32 storage, CG projection),
                                else it runs as MIXED; ACS_PREC_FP64: FP64 correction CG     */
    double cg_eta;           /* inexact projection: CG stops once its error estimate
                                sqrt(r' J^-1 r) <= eta * ||s_l - s_{l-1}||, eta starting at
                                cg_eta (default 0.3) and shrunk tenfold whenever the step
                                norm grows between rescalings; iterations that rescale
                                solve to the floors                                            */
    double cg_tol;           /* ... or <= cg_tol * ||s_l||; default 1e-12                     */
    int32_t cg_max_iter;     /* CG iterations per correction solve; default 500               */
    int32_t cg_refine;       /* correction solves per iteration, each from a fresh FP64
                                residual (mixed-precision refinement rounds); default 1, <= 8  */
    void* cuda_stream;       /* cudaStream_t to run on; NULL = the handle's own stream        */
    int32_t device;          /* CUDA device ordinal; default 0                                 */
    int32_t projection;      /* how the projection onto range((A O)') is applied:
                                ACS_PROJ_AUTO (default): the cached operator when
                                m <= dense_max_m, else CG with the switch below (for every
                                m <= 16384 when every row of A holds every column, nnz = m n);
                                ACS_PROJ_CG;
                                ACS_PROJ_DENSE: the cached operator whenever m <= 4096 (16384
                                with full rows, whose M is assembled by a tiled FP64 product).
                                The cached operator is
                                the FP64 Cholesky factor of M = (A O)(A O)', formed at every
                                rescaling, with L^{-1} kept so that each iteration's solve is
                                exact up to rounding (two dense products); a factorisation
                                that fails (M singular) switches that solve to CG          */
    int32_t dense_max_m;     /* largest m for the cached operator from the first iteration
                                under ACS_PROJ_AUTO; default 512, at most 4096                 */
    int32_t dense_switch_max_m; /* ACS_PROJ_AUTO, dense_max_m < m <= this: start with CG and
                                switch to the cached operator once the CG iterations since the
                                last rescaling exceed the cost of one factorisation counted in
                                CG iterations (0.3 m^3 / nonzeros, measured on the GB300), and
                                at least 8 * dense_switch_cg; default 1024, at most 4096      */
    int32_t dense_switch_cg; /* default 40; 0 disables the switch                               */
    double extrapolation;    /* start of each projection solve: w + theta (w - w_prev) with
                                theta = extrapolation (the matching A_hat' w follows without a
                                matrix pass while O is fixed); 0 (default) starts from the
                                previous w.  Measured on the large LP: theta = 0.5 and 1 take
                                540 and 1670 iterations instead of 390 (the smaller starting
                                residual lets the inexact solve stop with a larger error)     */
    int32_t a_storage;       /* values of A read by the FP32 correction CG: ACS_STORE_FP32
                                (default) or ACS_STORE_BF16 (2 bytes a nonzero, rounded to
                                nearest even; the FP64 passes -- residual of the projection
                                system, update, KKT -- still read the FP64 values, so the
                                refinement converges to the same FP64 iterate)                 */
    int32_t col_block;       /* FP32 matrix passes of acs_solve (single-problem launch): the
                                columns are cut into blocks whose FP32 vector entries fit one
                                CTA's shared memory, and every pass gathers from the staged
                                block instead of from L2; each row's partial sums are added in
                                block order.  0: blocks of at most 49152 columns; k > 0: at
                                most k columns (smaller blocks, for tests); -1 (default): off,
                                every pass gathers from L2 (the batched launch's layout).
                                Not used with a_storage = ACS_STORE_BF16 or when the cached
                                operator runs from the first iteration                         */
    double outer32_tol;      /* ACS_PREC_FP32: KKT level at which the outer products return
                                to FP64; default 1e-5                                          */
    int32_t splitting;       /* ACS_SPLIT_DR (default): the iteration of Algorithms 1-2,
                                Douglas-Rachford splitting of f = indicator of K and
                                g = c'x + indicator{Ax = b} (Section III-B);
                                ACS_SPLIT_ADMM: the ADMM of Section III-B for the same f, g
                                with penalty mu, run as Douglas-Rachford with the two proximal
                                steps swapped on zeta = x1 + z_admm/mu (one projection solve an
                                iteration, as for DR).  x is ADMM's x1 = proj_K(a) for the
                                reflection a = 2 prox_g(zeta) - zeta, y the multiplier of
                                Ax = b, s the state zeta, which starts where DR's s does:
                                (1 - mu) e from x = z = e, for mu = 1 the textbook start
                                x2 = z_admm = 0.  Needs L empty (cond_first = 0, no cond_list):
                                ADMM's x = proj_K(a) and z = proj_K(-a)/mu are exactly
                                complementary, so the ratio o of Algorithm 2 step 8 is 0, inf
                                or nan on every coordinate and the rescaling has nothing to
                                work with; other schedules give ACS_ERR_ARG                   */
    double polish_tol;       /* LP crossover polish inside acs_solve (K = R+^n; see acs_polish):
                                0 (default) = off.  With polish_tol > tol, acs_solve iterates
                                until every KKT residual is <= polish_tol and polishes; if the
                                polished point meets tol the solve ends there (ACS_SOLVED),
                                else the iteration resumes from its state (the scaling, the
                                multiplier and x, z as they were: as if uninterrupted) and
                                the polish is tried again at a ten times
                                lower level, until the iteration itself reaches tol.  These
                                polishes need only meet tol: their solves stop at 1e-3 tol /
                                polish_tol of their first residual (acs_polish itself goes
                                down to the rounding floor).  Only the
                                blocking acs_solve does this; acs_solve_async and the batched
                                and served forms ignore it.  Problems with Lorentz cones of
                                size >= 2 and polish_tol > 0 are rejected (ACS_ERR_ARG)        */
} acs_settings;

enum { ACS_SPLIT_DR = 0, ACS_SPLIT_ADMM = 1 };

enum { ACS_STORE_FP32 = 0, ACS_STORE_BF16 = 1 };

enum { ACS_PROJ_AUTO = 0, ACS_PROJ_CG = 1, ACS_PROJ_DENSE = 2 };

/* Fill *s with the defaults listed above.  Returns ACS_SOLVED or ACS_ERR_ARG. */
int acs_settings_default(acs_settings* s);

/*
 * Create a problem on the device.  Section II, Eq. (1).
 *   m, n        : A is m x n, m >= 1, n >= 1.
 *   row_ptr     : int64[m+1], row_ptr[0] = 0, non-decreasing, row_ptr[m] = nnz < 2^31.
 *   col         : int32[nnz], column indices in [0, n), strictly increasing in each row.
 *   val         : double[nnz].
 *   b           : double[m];  c : double[n].
 *   n_orthant   : number of leading nonnegative-orthant coordinates (>= 0).
 *   n_soc, soc_dims : Lorentz cones of sizes soc_dims[i] >= 2 following the orthant;
 *                 n_orthant + sum(soc_dims) must equal n.
 *   settings    : may be NULL for the defaults.
 *   out         : receives the handle (NULL on failure).
 * Every row of A must be nonempty.  The pseudoinverse of Algorithm 1 step 2
 * asks for A of full row rank; linearly dependent rows with a consistent b
 * are still solved (the cached operator drops the dependent direction, CG
 * stays in the range of M).  With an inconsistent b the problem is
 * infeasible and acs_solve ends with ACS_ERR_FACTOR, ACS_ERR_NUMERICAL or
 * ACS_MAX_ITER, never ACS_SOLVED.
 * Errors: ACS_ERR_ARG, ACS_ERR_CSR, ACS_ERR_CONES, ACS_ERR_OOM, ACS_ERR_CUDA.
 */
int acs_problem_create(int32_t m, int32_t n, const int64_t* row_ptr, const int32_t* col,
                       const double* val, const double* b, const double* c,
                       int32_t n_orthant, int32_t n_soc, const int32_t* soc_dims,
                       const acs_settings* settings, acs_problem** out);

/*
 * Run Algorithm 2 from the initial point x = z = e (the cone identity) until
 * every relative KKT residual is <= tol (ACS_SOLVED) or max_iter iterations
 * have run (ACS_MAX_ITER).  tol = 0 runs exactly max_iter iterations.
 * Residuals (all Euclidean, computed in FP64 with the FP64 copy of A):
 *   r_p   = ||Ax - b|| / (1 + ||b||)
 *   r_d   = ||A'y + z - c|| / (1 + ||c||)
 *   r_gap = |c'x - b'y| / (1 + |c'x| + |b'y|)
 *   r_cone= max(dist(x,K), dist(z,K)) / (1 + max(||x||, ||z||))
 * x, z are the iterates of Algorithm 2 steps 20-21 and y = w / mu, the
 * multiplier of the projection solve.  Blocks until done.
 */
int acs_solve(acs_problem* p, double tol, int32_t max_iter);

/* Same as acs_solve but returns as soon as the work is queued on the
 * handle's stream (ACS_SOLVED means "queued"); acs_get waits for it. */
int acs_solve_async(acs_problem* p, double tol, int32_t max_iter);

/*
 * Copy results to host buffers (any may be NULL): x[n], y[m], s[n] (the dual
 * slack, z of the paper), *iters, residuals[8] = {r_p, r_d, r_gap, r_cone,
 * obj_p, obj_d, CG iterations in total, iteration at which a mixed-precision
 * solve handed its correction solve over to FP64 (0 = never)}.  Waits for queued
 * work.  Returns the status of the last solve (>= 0) or an error.
 */
int acs_get(acs_problem* p, double* x, double* y, double* s, int32_t* iters, double* residuals);

/*
 * Checkpoint / warm start of the iteration state: s_dr[n] is the splitting
 * variable s of Algorithm 2 in the current scaled space, O[n] the diagonal
 * of O, w[m] the projection multiplier (mu * y), *l the iteration counter,
 * step[3] = {||s_l - s_{l-1}||, ||s_l||, current inexactness factor} used by
 * the inexact-projection rule (may be NULL: the next iteration then solves
 * to the CG floors and the factor restarts at cg_eta).
 * acs_set_state makes the next acs_solve continue from this state instead of
 * x = z = e (Algorithm 2 step 14 keeps progress across rescalings the same
 * way); a state taken after l iterations and resumed reproduces the
 * uninterrupted run.  All pointers are host pointers owned by the caller.
 * acs_get_state returns ACS_ERR_ARG after acs_polish until the next solve.
 */
int acs_get_state(acs_problem* p, double* s_dr, double* O, double* w, int32_t* l, double* step);
int acs_set_state(acs_problem* p, const double* s_dr, const double* O, const double* w, int32_t l,
                  const double* step);

/*
 * LP crossover polish of the last solve's iterate (K = R+^n only; not in the
 * paper, whose solver stops on its KKT test: an active-set alternative to
 * iterating on).  With B = {j : x_j > z_j}, the support of a strictly
 * complementary optimum:
 *   x~ = the orthogonal projection of x onto {u : u_j = 0 off B, A u = b}
 *      = x_B + A_B'(A_B A_B')^+ (b - A_B x_B) on B, 0 elsewhere;
 *   y~ = the least change of y with A_B' y~ = c_B in the metric of
 *        J = diag(A_B A_B') (J_ii = 1 on rows with no entry in B);
 *   z~ = c - A' y~.
 * At a nondegenerate vertex these are the vertex and its dual whatever x and
 * y were.  When |B| < m, y~ is fixed only up to null(A_B'): the CG path takes
 * the least change in the J-metric, the factored path the solution with no
 * component along the pivots it drops; both satisfy A_B' y~ = c_B.  Both solves run on the device in FP64, in up to `rounds` (1..8)
 * refinement rounds, each from a fresh FP64 residual: for m <= 4096,
 * M = A_B A_B' is assembled and factored once (the cached operator's
 * phases with O the indicator of B; a dependent row is dropped) and each
 * round applies its inverse factor; above that, or if the factorisation
 * fails, each round is a Jacobi-preconditioned CG from zero of at most
 * cg_max_iter iterations, down to the residual's rounding floor.  The polished
 * point replaces the iterate (acs_get then returns it and residuals[0..5]
 * are its own; the solve's status and iteration count stay) only if its
 * largest relative KKT residual is below the iterate's.
 * Returns ACS_SOLVED (replaced) or ACS_POLISH_KEPT (kept); ACS_ERR_ARG
 * before any solve, after a failed one, with Lorentz cones of size >= 2 or
 * rounds outside 1..8; ACS_ERR_OOM (the polish's buffers, 2n + 2m + 16
 * doubles and, for m <= 4096 on a handle without the cached operator,
 * 2 m^2, are allocated at the first call), ACS_ERR_CUDA,
 * ACS_ERR_DEVICE_TIMEOUT, ACS_ERR_NUMERICAL.  info (host, may be NULL):
 * info[7] = {|B|, CG iterations (factored M: corrections) of the x solve,
 * of the y solve, largest residual before, after, 1 if replaced, 1 if M was
 * factored}.  x, y, z are kept intact when the
 * polish is not taken, but the rest of the iteration state is used as
 * scratch: acs_get_state fails until the next acs_solve, which starts from
 * x = z = e (or from acs_set_state).  Blocks until done.
 */
int acs_polish(acs_problem* p, int32_t rounds, double* info);

/* Device memory of the single-problem API comes from a per-device cache:
 * the buffers of a destroyed handle (and the scratch of a create) are kept,
 * up to ACS_DEVICE_CACHE_MB megabytes (environment, default 4096), and reused
 * by later handles for requests of 80-100 % of a kept block's size, so that
 * repeated create/destroy cycles do not pay cudaMalloc/cudaFree.
 * acs_device_cache_trim returns the kept blocks of a device (-1: all) to the
 * driver; acs_device_cache_stats: out3 = {bytes kept, allocations served
 * from the cache, allocations that went to cudaMalloc} of a device. */
int acs_device_cache_trim(int32_t device);
int acs_device_cache_stats(int32_t device, int64_t* out3);

/* Release every device buffer of the handle (to the cache above).  NULL is ignored. */
void acs_problem_destroy(acs_problem* p);

/* Static string for a status code. */
const char* acs_status_string(int status);

/* Diagnostics.  acs_debug_counters: out6 = {A passes, A' passes, FP64 A passes,
 * FP64 A' passes, conditionings, FP64 iterations} of the last solve (the
 * benchmark's algorithmic-byte model counts matrix passes with these).
 * acs_problem_info: out8 = {m, n, nnz, stored entries of A and of A' after padding,
 * CTAs of the FP32 launch, CTAs of the FP64 launch, threads per CTA}. */
int acs_debug_counters(acs_problem* p, long long* out6);
/* Device time (ms) of the last persistent iteration launch, from CUDA events
 * recorded on the handle's stream around that launch; waits for it.  After an
 * acs_solve with polish_tol: the sum over its iteration launches.
 * acs_last_polish_ms: device time of the polish launches of the last solve
 * with polish_tol, or of the acs_polish calls since the last solve. */
int acs_last_launch_ms(acs_problem* p, double* ms);
int acs_last_polish_ms(acs_problem* p, double* ms);
/* Time of each phase of the persistent kernel in the last solve (ms, from
 * the device's global timer, barrier wait included) and how often it ran, in
 * the order: rescale-o, rescale-apply, b_tilde, q-refresh, abs_K, CG-rhs,
 * CG A' pass, CG A pass, CG vector step, update, KKT, cached-operator
 * factorisation, cached-operator correction, and for the column-blocked
 * passes the three phases that add up their partial sums: t = O^2 A'u of
 * the CG, the projection residual and the update of the FP32 outer passes,
 * then the cached operator's assembly of M and its inverse factor (the
 * factorisation entry covers the Cholesky steps).  n >= 18.  Returns the
 * number of phases written or an error. */
int acs_debug_phase_times(acs_problem* p, double* ms, long long* count, int32_t n);
/* Mean time (ns) of one grid-wide reduce-and-barrier of the persistent
 * kernel's launch shape, over n back-to-back barriers. */
int acs_debug_barrier_ns(acs_problem* p, int32_t n, double* ns);
int acs_problem_info(acs_problem* p, int32_t* out8);
/* Test of the failure path of the persistent kernel's grid barrier: one
 * grid-wide barrier of the solve's launch shape at which one CTA never
 * arrives.  The others' bounded waits (2 s) run out; they record
 * ACS_ERR_DEVICE_TIMEOUT and leave the kernel, which returns normally (no
 * trap; the context and the handle stay usable).  Returns the recorded
 * status and the time CTA 0 waited (ms). */
int acs_debug_barrier_timeout(acs_problem* p, double* waited_ms);
/* Host-only check of the preparation acs_problem_create does (no device
 * involved): the row relabelling and the sliced-ELLPACK image of A (which =
 * 0) or A' (which = 1) built for products run by `warps` warps.  A slice
 * holds 32 / g rows; entry k of local row r of slice q sits at
 * sptr[q] + 32 (k / g) + r g + (k mod g); padding entries have column 0 and
 * value 0.  Row r of the relabelled A is row perm[r] of the input; the rows
 * of A' list relabelled rows in increasing order.  The CSR is validated as
 * by acs_problem_create (all coordinates orthant).  info[4] = {rows, slices,
 * g, stored entries}; perm[m], sptr[slices + 1], slen[slices] (chunks of 32
 * entries per slice), col / val[stored] are written where not NULL (call
 * once with NULL arrays for the sizes).  Errors: ACS_ERR_ARG, ACS_ERR_CSR. */
/* The sliced-ELLPACK image of A (which = 0) or A' (which = 1) that a
 * problem holds on the device, read back: info[4] = {rows, slices, lanes
 * per row, stored entries}; sptr[slices + 1], slen[slices], col and val
 * (FP64) and v32 (FP32 copy, if the problem keeps one) [stored entries];
 * any array may be NULL.  Errors: ACS_ERR_ARG, ACS_ERR_CUDA. */
int acs_debug_images(acs_problem* p, int32_t which, int32_t* info, int32_t* sptr, int32_t* slen, int32_t* col,
                     double* val, float* v32);
/* Host-only check of the BF16 storage of A (a_storage = ACS_STORE_BF16):
 * out[k] = the BF16 bit pattern stored for the finite value v[k], i.e. its
 * FP32 value rounded to the nearest BF16 value, ties to even.  Errors:
 * ACS_ERR_ARG. */
int acs_debug_to_bf16(int64_t n, const double* v, uint16_t* out);
int acs_debug_sell(int32_t m, int32_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                   int32_t which, int64_t warps, int32_t* info, int32_t* perm, int32_t* sptr, int32_t* slen,
                   int32_t* out_col, double* out_val);
/* Host-only check of the column-blocked image acs_problem_create builds for
 * the FP32 passes (setting col_block): of the relabelled A (which = 0) or of
 * A' (which = 1), with blocks of at most width_limit (>= 4) columns, its
 * items dealt to `ctas` CTAs.  The columns are cut into nblocks blocks of
 * `width` columns (the last may be shorter); item = block * nsl + slice, a
 * slice being 32 rows; lane r of an item holds row
 * (slice / 64) * 2048 + rowid[item * 32 + r] (0xFFFF: no row), the rows of
 * each window of 2048 sorted by decreasing count of entries in the block
 * (stable); entry k of that row sits at sptr[item] + 32 k + r with the column
 * out_col - block * width and the FP32 value out_val; padding has column 0
 * and value 0; every item has at least one chunk of 32 entries, and bit
 * c mod 32 of cend[c / 32] is set exactly when chunk c (entries 32c ..
 * 32c + 31) is the last chunk of its item.  Items [cta_beg[c], cta_beg[c + 1])
 * go to CTA c.  info[6] = {rows, columns, width, nblocks, nsl, stored
 * entries}; perm[m] (the row relabelling, as acs_debug_sell),
 * sptr[nblocks * nsl + 1], rowid[32 * nblocks * nsl], out_col /
 * out_val[stored], cta_beg[ctas + 1], cend[stored / 1024 + 2] are written
 * where not NULL, and ipos[32 * nblocks * nsl], the inverse of rowid:
 * ipos[block * nsl * 32 + row] = the slot (slice within the window * 32 +
 * lane) that holds the row in that block.  Errors: ACS_ERR_ARG, ACS_ERR_CSR. */
int acs_debug_cbsell(int32_t m, int32_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                     int32_t which, int32_t width_limit, int32_t ctas, int64_t* info, int32_t* perm,
                     int32_t* sptr, uint16_t* rowid, uint16_t* out_col, float* out_val, int32_t* cta_beg,
                     uint32_t* cend, uint16_t* ipos);
/* Pass counters of the last solve: out[12] = {FP32 CG A passes, FP32 CG A'
 * passes, FP64 A passes, FP64 A' passes, rescalings, KKT checks, FP32 outer
 * A passes, FP32 outer A' passes, iteration at which the FP32 outer passes
 * ended (0 = never ran or did not end), iterations, CG iterations, iteration
 * of the FP32-to-FP64 CG hand-over}; n >= 12; with n >= 16 also {polishes
 * tried, polishes taken, their CG iterations (factored M: corrections), polishes
 * that factored M} of the last solve with polish_tol (or of acs_polish calls
 * since); with n >= 18 also {|B| of the last polish, stored entries of its
 * A_B (the rows of A on B's columns, which its CG passes read; 0 when it
 * factored M)}.  Counters of a polished solve add up all its segments.  Waits for
 * queued work.
 * acs_debug_layout: out[10] = {column-blocked layout in use, blocks of A,
 * width, stored entries, blocks of A', width, stored entries, dynamic shared
 * memory of the FP32 launch (bytes), stored entries of the sliced-ELLPACK A
 * and A'}; n >= 10; with n >= 12 also {slices of the sliced-ELLPACK A, of A'};
 * with n >= 14 also {bytes acs_problem_create copied host -> device, device ->
 * host}.
 * Both return the number of values written or an error. */
int acs_debug_pass_counts(acs_problem* p, int64_t* out, int32_t n);
int acs_debug_layout(acs_problem* p, int64_t* out, int32_t n);

/* Benchmarks (not part of a solve).
 * acs_bench_passes: device time (us) of one phase of the persistent kernel
 * on the problem's data, repeated `reps` times, each followed by a grid
 * barrier of the solve's launch shape (kind 9 times the barrier alone).
 * Kinds: 0 column-blocked A' pass of the CG (partial sums of A'u), 1 its
 * combine (t = O^2 A'u and u'Mu), 2 column-blocked A pass, 3 CG vector step
 * with the A pass's combine, 4 / 5 / 6 the same CG phases on the L2-gather
 * layout (FP32 values; only with col_block = -1), 7 FP64 projection-residual
 * pass over A, 8 FP64 pass over A', 9 barrier, 10 abs_K, 11 KKT residuals,
 * 12 / 13 FP32 outer projection residual (pass, combine), 14 / 15 FP32 outer
 * update (pass, combine), 16 / 17 the staging of the column-blocked A pass
 * alone (from an FP32 / an FP64 vector), 18 the column-blocked A' pass without
 * its gathers, 19 without its staging, 20 / 21 each CTA's entries of the A'
 * image read as one linear stream (columns and values / values only)
 * (diagnostics: the values they produce are meaningless).  smem_bytes: dynamic shared memory of the launch
 * (< 0: the solve's; more shrinks the L1 cache the same way a wider block
 * would; at least the solve's, except for kinds 18, 20 and 21, which read no
 * shared memory);
 * at most 196608.  The iterate state is left undefined: the next
 * acs_solve starts from x = z = e.  Errors: ACS_ERR_ARG, ACS_ERR_CUDA.
 * acs_bench_gather: random 4-byte gathers per second over the whole device
 * from a vector of `entries` floats (a power of two, 32 .. 2^24): mode 0
 * default loads, 1 L2-only loads, 2 read-only path, 3 from a copy in shared
 * memory (entries <= 49152); one CTA of 1024 threads per SM, 8 independent
 * gathers in flight per thread, `steps` rounds.  Allocates and frees its own
 * device buffers.  Errors: ACS_ERR_ARG, ACS_ERR_OOM, ACS_ERR_CUDA. */
int acs_bench_passes(acs_problem* p, int32_t kind, int32_t reps, int32_t smem_bytes, double* us_per_rep);
int acs_bench_gather(int32_t device, int64_t entries, int32_t mode, int32_t steps, double* gathers_per_s);

/*
 * KKT residuals of a caller-supplied point, for callers that cannot allocate
 * device memory (the paper has no counterpart; it is a service of this
 * library).  It allocates nothing: the caller passes every input and the
 * output in device memory it already owns, and the temporary data live in
 * one file-scope device array of fixed size, held by every GPU that loads the
 * library until the process exits.  Computes, in FP64 and in the order of
 * acs_get's residuals[0..5]: r_p, r_d, r_gap, r_cone, c'x, b'y (definitions
 * at acs_solve).
 *   m, n            : A is m x n, 1 <= n <= 1,048,576 (larger n: ACS_ERR_LIMIT);
 *                     the array is 8.06 MiB (n doubles for A'y plus 1024 x 8
 *                     block partials).
 *   row_ptr, col, val : DEVICE CSR of A: int32[m+1], int32[nnz], double[nnz].
 *   b[m], c[n], x[n], y[m], z[n] : DEVICE vectors (z is the dual slack).
 *   n_orthant, n_soc, soc_offsets : cones as in acs_problem_create, with
 *                     soc_offsets a DEVICE int32[n_soc+1] array of absolute
 *                     start offsets (soc_offsets[0] = n_orthant, increasing,
 *                     last = n).  The offsets live on the device and are not
 *                     checked (that would need a copy back to the host): a
 *                     malformed array makes the kernels read x and z out of
 *                     bounds.  Likewise row_ptr and col must describe a valid
 *                     CSR of A with columns in [0, n).
 *   residuals       : DEVICE double[6], written asynchronously.
 *   cuda_stream     : stream to run on (NULL = legacy default stream).
 * The call is asynchronous: results are ready when the stream reaches them.
 * Every call looks up the array's device address in the current context (a
 * host-side query that allocates nothing; the first one in a context loads
 * the library's device code), so the entry point stays valid after
 * cudaDeviceReset; make the first call in a context before any stream
 * capture.  An error left by an earlier, unrelated launch is cleared at the
 * start of the call and not reported by it.
 * Every call clears the part of the array it accumulates into; calls that
 * overlap on the GPU share the array and race, so order them.  The A'y part
 * is accumulated with atomic adds, so r_d may differ in its last bits from
 * call to call.  Errors: ACS_ERR_ARG, ACS_ERR_LIMIT, ACS_ERR_CUDA.
 */
int acs_kkt_residuals_noalloc(int32_t m, int32_t n, const int32_t* row_ptr, const int32_t* col,
                              const double* val, const double* b, const double* c, const double* x,
                              const double* y, const double* z, int32_t n_orthant, int32_t n_soc,
                              const int32_t* soc_offsets, double* residuals, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Batched solves: many independent programs of uneven sizes in one
 * persistent launch (replayed from a captured CUDA graph).
 *
 * Every member is an instance of Eq. (1) solved by Algorithm 2 exactly as
 * acs_solve does (same settings for all members).  The launch is split into
 * fixed teams of CTAs; a team takes the next member (largest first), runs
 * its whole solve with team-local barriers and reductions (no grid-wide
 * synchronisation), then takes the next.  Members that share one A (same
 * pattern and values) keep a single device copy of it.
 * ------------------------------------------------------------------------ */
typedef struct acs_batch acs_batch;

typedef struct {
    int32_t m, n;            /* as in acs_problem_create                                  */
    const int64_t* row_ptr;  /* host CSR of A (ignored when share_A_with >= 0)            */
    const int32_t* col;
    const double* val;
    const double* b;         /* host, [m]                                                 */
    const double* c;         /* host, [n]                                                 */
    int32_t n_orthant, n_soc;
    const int32_t* soc_dims; /* host, [n_soc]                                             */
    int32_t share_A_with;    /* -1, or the index of an EARLIER member whose A this member
                                reuses (same m and n; the caller guarantees equal data)   */
} acs_instance;

typedef struct {
    int32_t threads_per_cta; /* 256, 512 or 1024                                          */
    int32_t team_ctas;       /* CTAs per team: 1, 2, 4 or 8                               */
} acs_batch_mapping;

/*
 * Create a batch of `count` >= 1 members (host data, copied; the pointers are
 * read only during the call).  settings: as for acs_problem_create (NULL =
 * defaults), shared by all members.  mapping: NULL = {1024, 1} until
 * acs_batch_autotune picks one.
 * Errors: ACS_ERR_ARG (also a bad share_A_with), ACS_ERR_CSR, ACS_ERR_CONES
 * (the first failing member's code; *bad_member receives its index if not
 * NULL), ACS_ERR_OOM, ACS_ERR_CUDA.
 */
int acs_batch_create(int32_t count, const acs_instance* members, const acs_settings* settings,
                     const acs_batch_mapping* mapping, acs_batch** out, int32_t* bad_member);

/* Solve every member from x = z = e to tol / max_iter (as acs_solve).  The
 * first call with a given (tol, max_iter, mapping) captures the reset and
 * the persistent launch into a CUDA graph; later calls replay it.  Blocks
 * until done and returns ACS_SOLVED if every member was solved, ACS_MAX_ITER
 * if some reached the limit, else the first member error.  The _async form
 * only queues the work on the batch's stream. */
int acs_batch_solve(acs_batch* b, double tol, int32_t max_iter);
int acs_batch_solve_async(acs_batch* b, double tol, int32_t max_iter);

/* Results of member i (as acs_get; any pointer may be NULL).  Waits for
 * queued work.  Returns that member's status. */
int acs_batch_get(acs_batch* b, int32_t i, double* x, double* y, double* s, int32_t* iters,
                  double* residuals);

/* Status, iterations and residuals[8] (as acs_get) of every member at once:
 * status[count], iters[count], residuals[8 * count]; any may be NULL. */
int acs_batch_results(acs_batch* b, int32_t* status, int32_t* iters, double* residuals);

/* Time every candidate mapping (threads per CTA in {256, 512, 1024} x team
 * sizes in {1, 2, 4}) on a truncated solve of the whole batch (max_iter
 * iterations, no stopping test), keep the fastest and return it in *chosen
 * (may be NULL); ms[9] (may be NULL) receives each candidate's time in the
 * order threads-major, team-minor (negative = not launchable). */
int acs_batch_autotune(acs_batch* b, int32_t max_iter, acs_batch_mapping* chosen, double* ms);

/* Set the mapping explicitly (invalidates the captured graph). */
int acs_batch_set_mapping(acs_batch* b, const acs_batch_mapping* mapping);

/* Device time (ms) of the last batched launch (graph replay), from CUDA
 * events on the batch's stream; waits for it. */
int acs_batch_last_ms(acs_batch* b, double* ms);

/* out8 = {members, distinct matrices, sum m, sum n, sum of stored nonzeros of
 * distinct matrices, teams of the current mapping, CTAs, 1 if the last solve
 * was replayed from a CUDA graph}.  counters6 (may be NULL): acs_debug_counters
 * summed over members. */
int acs_batch_info(acs_batch* b, long long* out8, long long* counters6);

/* Pass counters of every member's last solve: out[8 * count], per member
 * {A passes, A' passes (FP32 or FP64 correction CG), FP64 A passes, FP64 A'
 * passes, rescalings, KKT checks, cached-operator corrections, cached-operator
 * factorisations}.  Waits for queued work. */
int acs_batch_counters(acs_batch* b, long long* out);

/* Device time (ms, the team's global timer from its first to its last
 * barrier on the member, barrier waits included) each member's last solve
 * took: ms[count].  Waits for queued work. */
int acs_batch_member_ms(acs_batch* b, double* ms);

/* Per-phase device times (ms) and counts of member i's last solve, or summed
 * over all members for i = -1, in the order of acs_debug_phase_times; n >= 18.
 * Returns the number of phases written or an error. */
int acs_batch_phase_ms(acs_batch* b, int32_t i, double* ms, long long* count, int32_t n);

void acs_batch_destroy(acs_batch* b);

/* Host-only check of the preparation acs_batch_create does before it uses
 * the device: validation, relabelling and images of every distinct A, and
 * the host image of the batch's static device region (matrices, b, c, cone
 * offsets, member order) at its final offsets.  *hash = FNV-1a of that image,
 * *static_bytes = its size.  Errors: those of acs_batch_create's host
 * checks, with *bad_member as there. */
int acs_debug_batch_image(int32_t count, const acs_instance* members, const acs_settings* settings,
                          uint64_t* hash, int64_t* static_bytes, int32_t* bad_member);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of independent solves.
 *
 * A worker thread owned by the server admits submitted requests into a
 * device memory pool of a fixed budget (a request waits while it does not
 * fit, or while every slot is taken), keeps each admitted request's data and
 * iterates on the device, and runs rounds: one persistent team launch over
 * every admitted request, time-sliced by a device-side deadline at which
 * each request pauses at the end of an iteration.  A paused request resumes
 * from its device state in the next round exactly where it stopped, so its
 * result is the one it has when solved alone in a batched launch of the
 * same mapping.  When fewer requests are admitted than the launch has
 * CTAs, every request gets a team of its own sized by its work (so a few
 * large requests spread over the whole GPU); otherwise teams of the
 * configured size take requests from a queue.  Finished requests leave
 * between rounds, freeing their slot and memory for waiting ones, so
 * requests that arrive while others are on the GPU join the next round.
 * Requests larger than large_nnz stored entries run alone, between rounds,
 * on the whole GPU (the single-problem launch).  Each request is solved by
 * Algorithm 2 like acs_solve, with the server's settings and its own tol /
 * max_iter.
 * ------------------------------------------------------------------------ */
typedef struct acs_server acs_server;

typedef struct {
    int64_t budget_bytes;    /* device memory for admitted requests; default 4 GiB          */
    int32_t max_active;      /* slots (requests admitted at once); default 2048             */
    double round_ms;         /* time slice of one round; default 2 ms                       */
    int64_t large_nnz;       /* requests whose A has more nonzeros run alone on the whole
                                GPU; default 8388608                                         */
    int32_t threads_per_cta; /* mapping of the rounds (as acs_batch_mapping); default 256   */
    int32_t team_ctas;       /* default 1                                                    */
    int64_t long_nnz;        /* requests whose A has more nonzeros are "long": while long and
                                short requests are both admitted, rounds alternate between the
                                two classes with equal time for each, so that short requests do
                                not wait idle for a long request's iteration (the deadline is
                                checked at the end of an iteration); 0 = one class; default
                                262144                                                         */
    int32_t adaptive_teams;  /* 1 (default): work-sized teams while fewer requests than CTAs
                                are admitted; 0: always queued teams of team_ctas CTAs, so
                                that every request's arithmetic (reduction order included) is
                                the same in every round and a served result equals, bit for
                                bit, the request solved alone by acs_batch_solve with the same
                                mapping                                                        */
} acs_server_config;

int acs_server_config_default(acs_server_config* cfg);

/* settings: shared by all requests (NULL = defaults; cuda_stream is ignored,
 * the server owns its stream).  Errors: ACS_ERR_ARG, ACS_ERR_OOM (the budget
 * cannot be allocated), ACS_ERR_CUDA. */
int acs_server_create(const acs_settings* settings, const acs_server_config* cfg, acs_server** out);

/* Validate and prepare a request on the calling thread (host work only) and
 * queue it; returns at once with *id.  The acs_instance's share_A_with must
 * be -1.  per_request (may be NULL): this request's mu, t, cond_first,
 * cond_period and check_every (e.g. the SOCP schedule t = 1.7, L = {200,
 * 300, ...} for a request with Lorentz cones, the LP one for an LP); every
 * other setting is the server's, and its cond_list must be empty.
 * Errors: ACS_ERR_ARG, ACS_ERR_CSR, ACS_ERR_CONES, ACS_ERR_LIMIT (the request
 * can never fit the budget).  Thread-safe. */
int acs_server_submit(acs_server* s, const acs_instance* req, double tol, int32_t max_iter,
                      const acs_settings* per_request, int64_t* id);

/* *done = 1 once request id has finished.  Thread-safe. */
int acs_server_poll(acs_server* s, int64_t id, int32_t* done);

/* Block until request id has finished or timeout_s has passed (< 0: no
 * limit).  Returns the request's status, ACS_ERR_DEVICE_TIMEOUT if the wait
 * timed out, or ACS_ERR_ARG for an unknown id (also when another thread's
 * acs_server_result took the request during the wait).  Thread-safe. */
int acs_server_wait(acs_server* s, int64_t id, double timeout_s);

/* Results of a finished request (as acs_get; any pointer may be NULL) and
 * its latency (ms) from the entry of acs_server_submit (host preparation
 * included) to the moment its results were in host memory; then the server
 * forgets the request.  Returns its status, or ACS_ERR_ARG for an unknown or
 * unfinished id.  Thread-safe. */
int acs_server_result(acs_server* s, int64_t id, double* x, double* y, double* sl, int32_t* iters,
                      double* residuals, double* latency_ms);

/* out[10] = {rounds, requests admitted, requests finished, requests active,
 * pool bytes in use, peak pool bytes, requests run alone (large), requests
 * waiting, mean ms per round, mean active requests per round}. */
int acs_server_stats(acs_server* s, double* out);

/* Finish every submitted request, stop the worker, release everything. */
void acs_server_destroy(acs_server* s);

/* Host-only checks of the serving loop's bookkeeping (no device involved).
 * acs_debug_assign_teams: the work-sized teams of a round with n <= grid
 * requests of the given work (> 0): cta[3 * grid] = per CTA the request's
 * position (-1 = idle), its rank in the team and the team size.
 * acs_debug_arena: runs ops on a first-fit pool of cap bytes: ops[k] > 0
 * allocates ops[k] bytes (offsets[k] = its offset, or -1 if it did not fit),
 * ops[k] < 0 frees the block of op -ops[k]-1; used_peak[2] = bytes in use at
 * the end and the peak (blocks are rounded up to 256 bytes).
 * Both return ACS_SOLVED, or ACS_ERR_ARG for n outside [1, grid], a work
 * <= 0, a NULL pointer, or a free of a later, failed or already freed block. */
int acs_debug_assign_teams(int32_t n, const double* work, int32_t grid, int32_t* cta);
int acs_debug_arena(int64_t cap, int32_t nops, const int64_t* ops, int64_t* offsets, int64_t* used_peak);

/* Library version string. */
const char* acs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ACS_H */
