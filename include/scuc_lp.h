/*
 * scuc_lp.h -- C ABI of the B300 (sm_103a) library that solves SCUC LP
 * relaxations with the restarted Halpern Peaceman-Rachford (HPR) iteration
 * and runs the logic-driven fixing + bound propagation between relaxations.
 *
 * Paper: "Successive Fixing for Large-Scale SCUC Using First-Order Methods".
 *   LP form ............ Sec. 3, Eq. 8:  min mu^T x  s.t.  A x >= theta,
 *                        x in K = [x^L, x^U].  Here the row set is a box
 *                        lo <= A x <= hi given by a sense per row.
 *   Iteration .......... Sec. 3, Eq. 9 (x-, y-, z-steps, reflection,
 *                        Halpern anchoring); lambda = lambda_max(A A^T) by
 *                        the power method (Sec. 3, text after Eq. 9).
 *   Stopping ........... KKT residual map of Theorem 1 (normalised).
 *   Scaling ............ Sec. 3.A: Pock-Chambolle diagonal scaling and
 *                        normalisation of bounds and costs (Ruiz off).
 *   FP32 matvecs ....... Sec. 3.B: low-precision arithmetic for the core
 *                        steps; here the matvecs only, with FP64 iterates,
 *                        reductions and a final FP64 phase.
 *   Round / fixing ..... Sec. 4.1, Round operator and Algorithm 1.
 *   Presolve ........... Sec. 4.2, Algorithm 2 (MILP-/LP-Presolve): bound
 *                        propagation and removal of fixed columns and
 *                        redundant rows.
 *   Second algorithm ... restarted PDHG with ergodic averaging on the same
 *                        steps (the method HPR improves on, Sec. 3), and
 *                        infeasibility detection with certificates.
 *   Filtering .......... the transmission-filtering loop of Fig. 1: violated
 *                        pool rows found on the device and appended.
 *
 * Conventions (all entry points):
 *   - Return value is an scuc_err code; SCUC_OK on success.  On failure
 *     scuc_last_error() gives a message (thread-local, valid until the next
 *     call on the same thread).  Solver outcomes go to info->status.
 *   - Every pointer argument is caller-owned and never retained.  Host
 *     arrays are read (or written) during the call only.  Device pointers
 *     are used only where a parameter says so.
 *   - A handle owns its device copies; it is not thread-safe; all its work is
 *     ordered on the CUDA stream given at creation (NULL = legacy default
 *     stream) on the device that was current at creation.
 *   - Invalid input (sizes, unsorted or out-of-range column indices, NaN,
 *     lo > hi, xl > xu) returns SCUC_E_INVALID before any launch.
 *   - Sizes: m, n < 2^31 and nnz < 2^31 (32-bit indices on the device).
 *   - No entry point synchronises the whole device; each solve synchronises
 *     its stream before returning.  Solves allocate no pinned host memory;
 *     creating a handle allocates a small pinned control block and
 *     page-locks the caller's matrix arrays (>= 64 MiB each) for the
 *     duration of their copy, releasing them before it returns.
 */
#ifndef SCUC_LP_H
#define SCUC_LP_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scuc_lp scuc_lp;

enum scuc_err {
  SCUC_OK = 0,
  SCUC_E_INVALID = 1,        /* bad argument or malformed input             */
  SCUC_E_CUDA = 2,           /* a CUDA runtime call failed                  */
  SCUC_E_OOM = 3,            /* device allocation failed                    */
  SCUC_E_DEVICE_TIMEOUT = 4, /* a kernel's bounded wait ran out (the warm-
                                start network's tcgen05 GEMM)               */
  SCUC_E_INFEASIBLE = 5      /* propagation proved the fixed model infeasible */
};

enum scuc_status {
  SCUC_ST_OPTIMAL = 0,       /* max(r_p, r_d, gap) <= tol                   */
  SCUC_ST_ITER_LIMIT = 1,
  SCUC_ST_TIME_LIMIT = 2,
  SCUC_ST_NUMERICAL = 3,     /* NaN/Inf appeared in a residual              */
  SCUC_ST_FALLBACK_COLD = 4, /* warm start rejected, solved from cold start */
  SCUC_ST_PRIMAL_INFEASIBLE = 5, /* infeas_tol > 0: y_out holds a Farkas ray  */
  SCUC_ST_DUAL_INFEASIBLE = 6    /* infeas_tol > 0: x_out holds a direction of
                                    unbounded descent (primal unbounded)    */
};

enum scuc_algo {
  SCUC_ALGO_HPR = 0,         /* restarted Halpern PR iteration (Eq. 9)      */
  SCUC_ALGO_PDHG_AVG = 1     /* restarted PDHG with ergodic averaging: the
                                same two steps without the Halpern step;
                                checks and restarts on the running average
                                of the restart cycle                         */
};

enum scuc_precision {
  SCUC_FP64 = 0,             /* FP64 matvecs                                */
  SCUC_MIXED = 1             /* FP32 matvecs + FP32 accumulation, FP64
                                iterates/reductions/restarts, FP64 final
                                phase (Sec. 3.B)                             */
};

/* Solver parameters.  scuc_default_params() fills the defaults given in the
 * comments; the restart and sigma rules are the readings of "adaptive sigma
 * updates and restart schemes" (Sec. 3, after Theorem 1) described with
 * scuc_lp_solve.                                                         */
typedef struct {
  double tol;             /* 1e-4: stop when max(r_p, r_d, gap) <= tol      */
  int64_t max_iter;       /* 1e6 (rounded up to a multiple of check_every)  */
  double time_limit_s;    /* 3600 (wall time, checked at KKT checks)        */
  int32_t check_every;    /* 64: iterations between KKT/restart checks      */
  int32_t precision;      /* SCUC_FP64                                      */
  int32_t use_scaling;    /* 1: Pock-Chambolle + normalisation (Sec. 3.A);
                             2: 10 Ruiz passes first (the HPR-LP default
                             that Sec. 3.A replaces); 0: none               */
  double sigma0;          /* 1.0: initial primal step sigma                 */
  double lambda_in;       /* 0: run the power method; > 0: use this value   */
  double lambda_safety;   /* 1.01: lambda = safety * power estimate         */
  int32_t power_max_iter; /* 500                                            */
  double power_tol;       /* 1e-4 relative change of the estimate           */
  uint64_t power_seed;    /* 0x5EED: start q_j = 0.5 + U01(SplitMix64(seed +
                             (j+1) * 0x9E3779B97F4A7C15))                   */
  double restart_suff;    /* 0.2 */
  double restart_nec;     /* 0.8 */
  double restart_long;    /* 0.2 */
  double polish_factor;   /* 1: MIXED switches to FP64 matvecs at kkt <=
                             max(factor*tol, polish_floor), or on a stall;
                             FP32 matvecs reach 1e-4, 1e-5 and 1e-6 on the
                             13k-bus LP in as many iterations as FP64, so
                             with factor 1 and tol >= polish_floor the whole
                             solve runs FP32 matvecs; 10 polishes the last
                             decade                                        */
  int32_t polish_stall;   /* 200: ... or after this many checks without a
                             10% improvement of the best KKT measure (HPR's
                             KKT measure has plateaus of dozens of checks
                             that FP64 matvecs do not shorten)              */
  int32_t use_graph;      /* 1: replay each check period as a CUDA graph    */
  int32_t profile;        /* 1: time the two SpMV kernels with CUDA events  */
  int32_t device_ptrs;    /* 1: x0/y0 and x/y/z_out of scuc_lp_solve are
                             device pointers on the handle's device         */
  int32_t restart_ref;    /* reference rho0 of the restart tests: 0 = rho at
                             the first check of the cycle; 1 = rho at the
                             check that made the last restart               */
  int32_t restart_metric; /* rho of the restart tests: 0 = sqrt(||dx||^2/sigma
                             + lambda sigma ||dy||^2) with dx = x_bar - x,
                             dy = y_bar - y; 1 = the same plus 2<A dx, dy>
                             (the norm in which the iteration is
                             nonexpansive); 2 = KKT error                   */
  int32_t sigma_update;   /* 1: sigma update at restarts; 0: keep sigma0    */
  int32_t algo;           /* SCUC_ALGO_HPR                                  */
  double infeas_tol;      /* 0: off; > 0: at every check, declare the LP
                             primal infeasible when y_bar - y is a Farkas
                             ray, or unbounded when x_bar - x is a descent
                             direction in the recession cone, each with
                             relative violation <= infeas_tol (1e-8 is a
                             sound choice); two extra FP64 SpMVs per check */
  int32_t spmv_layout;    /* 0: the primal step's A^T y runs on a sliced ELL
                             copy of A^T (slices of 32 columns of A, one per
                             lane) when the handle has one (every column of
                             A holds <= 4096 nonzeros); 1: on the CSR
                             partition, like every other product          */
  int32_t split_steps;    /* scuc_lp_solve with spmv_layout 0 (batches keep
                             separate launches): 0: on plain (non-check)
                             iterations the primal update runs in the sliced
                             ELL product's launch (iterates bit-identical to
                             1), and, when A has rows above 512 nonzeros,
                             the dual step runs A's other rows on a sliced
                             ELL copy of A in the launch of the long rows'
                             chunk warps, their updates fused (their sums in
                             row order: iterates equal to rounding); 1: the
                             product and the update as separate launches on
                             the CSR partition of A, as on check
                             iterations                                   */
  double polish_floor;    /* 1e-6: MIXED moves to FP64 matvecs once kkt <=
                             this (the accuracy FP32 matvecs were measured to
                             reach without extra iterations), so tolerances
                             below it get an FP64 final phase              */
} scuc_solve_params;

typedef struct {
  int32_t status;         /* scuc_status                                    */
  int32_t restarts;
  int64_t iters;          /* total HPR iterations                           */
  int64_t iters_fp32;     /* of which with FP32 matvecs                     */
  int32_t power_iters;
  int32_t nlog;           /* entries in the check log (scuc_lp_get_log)     */
  double kkt, rp, rd, gap;/* at the returned point (unscaled LP)            */
  double pobj, dobj;      /* primal and dual objective (unscaled LP)        */
  double lambda, sigma;   /* lambda used, final sigma                       */
  double beta, gamma;     /* normalisation factors of Sec. 3.A              */
  double setup_ms;        /* scaling + power method                         */
  double solve_ms;        /* iterations (wall, stream-synchronised)         */
  /* profile = 1: summed CUDA-event time and launch counts of the SpMV
   * kernels (dual step = A x_tilde, primal step = A^T y)                  */
  double ms_dual_spmv, ms_primal_spmv;
  int64_t n_dual_spmv, n_primal_spmv;
  /* the part of the above that ran with FP32 matvecs (MIXED)              */
  double ms_dual_spmv_f32, ms_primal_spmv_f32;
  int64_t n_dual_spmv_f32, n_primal_spmv_f32;
  int64_t launches;       /* kernels launched by this solve                 */
  int64_t warm_iters;     /* scuc_lp_solve_warm: iterations of a rejected
                             warm run (included in iters); 0 otherwise     */
  int64_t ref_iters;      /* scuc_lp_solve_warm: iterations of the cold
                             reference period (included in iters)         */
  double cold_first_kkt;  /* scuc_lp_solve_warm: KKT measure at the cold
                             start's first check; 0 otherwise             */
} scuc_solve_info;

typedef struct {
  int64_t iter;           /* total iterations at this check                 */
  int32_t restart;        /* 1 if the check restarted the Halpern cycle     */
  int32_t first;          /* 1 if first check of its cycle                  */
  double rp, rd, gap, pobj, dobj;
  double rho;             /* restart metric (scaled space)                  */
  double sigma;           /* sigma in force during the checked period       */
  int32_t fp64;           /* 1 if the period used FP64 matvecs              */
  int32_t pad;
} scuc_check_log;

/* Defaults listed in scuc_solve_params. */
void scuc_default_params(scuc_solve_params* p);

/* Create an LP  min c^T x  s.t.  row_i(A x) in [lo_i, hi_i], xl <= x <= xu
 * (Eq. 8).  Host CSR: row_ptr[m+1] (int64, row_ptr[0] = 0, nondecreasing),
 * col[nnz] (int32, strictly increasing within a row, in [0, n)), val[nnz]
 * (finite FP64).  c[n] finite; xl[n], xu[n] may be -INF / +INF.
 * sense[m]: 'G' (lo = rhs, hi = +INF), 'L' (lo = -INF, hi = rhs),
 * 'E' (lo = hi = rhs), 'R' (lo = rhs, hi = rhs + range, range >= 0).
 * range may be NULL when no row is 'R'.  cuda_stream: cudaStream_t or NULL.
 * All data are copied to the device of the current CUDA context; the
 * transposed matrix is built on the device.  *out receives the handle.   */
int scuc_lp_create(scuc_lp** out, int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                   const int32_t* col, const double* val, const double* c, const double* xl,
                   const double* xu, const char* sense, const double* rhs, const double* range,
                   void* cuda_stream);

/* Same with the row box given directly: lo[m], hi[m] (lo <= hi, +-INF). */
int scuc_lp_create_box(scuc_lp** out, int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                       const int32_t* col, const double* val, const double* c, const double* xl,
                       const double* xu, const double* lo, const double* hi, void* cuda_stream);

/* Dimensions of a handle. */
int scuc_lp_dims(const scuc_lp* lp, int32_t* m, int32_t* n, int64_t* nnz);

/* Storage of the matrix entries that the FP32 iteration products (Eq. 9
 * with FP32 matrix-vector products, Sec. 3.B) read, for byte accounting.
 * Valid after the handle's first solve with FP32 products (0 before).
 * out[8] (host):
 *   0  entries of A's chunked rows read with 16-bit column offsets
 *      (6 bytes each: FP32 value + offset from the chunk's first column)
 *   1  entries of A's chunked rows read with 32-bit columns (8 bytes)
 *   2  entries (incl. padding) of the sliced copy of A's other rows
 *      (8 bytes each)
 *   3  entries (incl. padding) of the sliced copy of A^T
 *   4  1 if that copy stores 16-bit row offsets (6 bytes per entry and a
 *      16-byte record per column), 0 if 32-bit rows (8 bytes per entry)
 *   5  lanes (columns incl. empty lanes) of the sliced copy of A^T
 *   6, 7  as 0, 1 for A^T's chunked columns
 * Returns SCUC_E_INVALID for a null handle or output.                    */
int scuc_lp_layout(const scuc_lp* lp, int64_t* out);

/* on = 1 (the default): FP32 products read the matrix's column (row)
 * indices as 16-bit offsets where the layout allows (scuc_lp_layout);
 * 0: 32-bit indices everywhere (the same sums: an A/B switch).  Set before
 * the handle's first solve; afterwards, or for on not 0/1, SCUC_E_INVALID.
 * This storage format is this library's, not the paper's.                */
int scuc_lp_set_index16(scuc_lp* lp, int32_t on);

/* Solve with restarted HPR (Eq. 9), or restarted PDHG with ergodic
 * averaging (p->algo).
 *  x0[n], y0[m]: optional warm start (NULL = cold start from x = Pi_K(0),
 *    y = 0); projected onto K and onto the sign pattern of the rows.
 *  x_out[n], y_out[m], z_out[n]: caller buffers (NULL allowed) receiving
 *    the last checked point (x_bar, y_bar, z_bar) in the unscaled LP; with
 *    status SCUC_ST_PRIMAL_INFEASIBLE y_out receives the unscaled Farkas
 *    ray u instead (sum_i (u_i > 0 ? lo_i : hi_i) u_i + sum_j (z_j > 0 ?
 *    xl_j : xu_j) z_j > 0 with z = -A^T u), with SCUC_ST_DUAL_INFEASIBLE
 *    x_out receives the direction d (c^T d < 0, A d and d in the recession
 *    cones of the row box and of K).
 *  Host or device pointers according to p->device_ptrs.
 *  Per iteration k (k counts iterations since the last restart, scaled
 *  problem, s = 1/(lambda sigma)):
 *    x_bar = Pi_K(x + sigma (A^T y - c));   z_bar = (x_bar - v)/sigma
 *    x_t   = 2 x_bar - x;                   y_bar = P_s(y - s A x_t)
 *    with P_s(r) = r + s Pi_[lo,hi](-r/s), i.e. Pi_+(y + s(theta - A x_t))
 *    for rows A x >= theta;  then x, y <- (anchor + (k+1)(2 bar - old))/(k+2).
 *  Every check_every iterations the KKT residuals r_p = ||Ax - Pi(Ax)|| /
 *  (1+||b||), r_d = ||c - A^T y - z|| / (1+||c||), gap = |p-d|/(1+|p|+|d|)
 *  are evaluated at (x_bar, y_bar, z_bar) of the unscaled LP, and the cycle
 *  restarts (anchor <- current point, k <- 0) on the first check with
 *  k >= restart_long * total, or on a later check with
 *  rho <= restart_suff*rho0, or rho <= restart_nec*rho0 and rho > rho_prev,
 *  or k >= restart_long*total; rho = sqrt(||x_bar-x||^2/sigma +
 *  lambda sigma ||y_bar-y||^2).  At a restart sigma <- sqrt(sigma *
 *  ||dx||/(sqrt(lambda) ||dy||)) with d the displacement since the last
 *  restart (skipped when either norm < 1e-10).
 *  SCUC_ALGO_PDHG_AVG: x, y <- x_bar, y_bar; the running averages
 *  (x_avg, y_avg) of the cycle's (x_bar, y_bar) (weights 1/(k+1)) are the
 *  checked point, z the reduced cost c - A^T y_avg where a finite bound
 *  lets it act (0 elsewhere); rho = the KKT error; a restart moves the
 *  iterate and the anchor to the average.
 *  info (may be NULL) receives the outcome; the check log is kept in the
 *  handle (scuc_lp_get_log).  Synchronises the handle's stream.         */
int scuc_lp_solve(scuc_lp* lp, const scuc_solve_params* p, const double* x0, const double* y0,
                  double* x_out, double* y_out, double* z_out, scuc_solve_info* info);

/* Copy up to cap entries of the last solve's check log into out (host);
 * *count receives the number copied.                                    */
int scuc_lp_get_log(const scuc_lp* lp, scuc_check_log* out, int32_t cap, int32_t* count);

/* Unscaled products on device buffers of the handle's device:
 * transpose = 0: out[m] = A in[n];  transpose = 1: out[n] = A^T in[m].
 * Uses the same SpMV kernels as the solver (FP64).                      */
int scuc_lp_matvec(scuc_lp* lp, int32_t transpose, const double* in_dev, double* out_dev);

/* Batch of LP solves: the successive-fixing rounds of many instances are
 * independent relaxations (Sec. 4, Algorithm 2), solved here together.
 * The LPs are laid out as one block-diagonal LP and each iteration of Eq. 9
 * is one launch over all of them; every LP keeps its own scaling (Sec.
 * 3.A), lambda, sigma, Halpern counter, restarts, precision phase and stop
 * test, so each follows the iteration of its own scuc_lp_solve (the same
 * checks and restart decisions; matvec sums may differ in rounding order).
 *  lps[count]: distinct handles on one device (SCUC_E_INVALID otherwise).
 *  p: as scuc_lp_solve (profile is ignored); NULL: defaults.  Only
 *    SCUC_ALGO_HPR without infeasibility detection (SCUC_E_INVALID
 *    otherwise).
 *  x_out[count], y_out[count], z_out[count]: NULL, or per-LP output
 *    pointers (each may be NULL), device or host per p->device_ptrs.
 *  infos[count]: per-LP results; setup_ms/solve_ms/launches are those of
 *    the whole batch.  Each handle's check log is replaced by its LP's.
 *  binfo (may be NULL): autotune is read (NULL: on); the chosen SpMV
 *    partition shapes and the batch timings are written.  Tuned shapes are
 *    kept for the process, keyed by precision and the LPs' sizes, and a
 *    later batch with the same key uses them without timing.
 * The call returns after all work has completed.                        */
typedef struct {
  int32_t autotune;        /* in: 1 = time candidate partition shapes       */
  int32_t ept_A, run_A;    /* out: entries per thread of list rows, shortest
                              staged run, for A                            */
  int32_t ept_T, run_T;    /* out: the same for A^T                         */
  int32_t candidates;      /* out: shapes timed                             */
  int32_t blocks_A, blocks_T;  /* out: blocks of one SpMV launch            */
  double setup_ms;         /* out: scaling, power methods, layout, tuning   */
  double tune_ms;          /* out: of which the partition tuning            */
  double solve_ms;         /* out: iterations                               */
  double total_ms;         /* out: whole call                               */
  int64_t launches;        /* out: kernels launched                         */
  int64_t periods;         /* out: check periods run                        */
  double scale_ms;         /* out: of setup_ms, every LP's scaling and power
                              method (queued on the LPs' own streams)      */
  int32_t tune_cached;     /* out: 1 = the shapes came from an earlier batch
                              of the same precision and LP sizes (no
                              timing this call)                            */
  int32_t reserved0;
} scuc_batch_info;

int scuc_lp_solve_batch(scuc_lp* const* lps, int32_t count, const scuc_solve_params* p,
                        double* const* x_out, double* const* y_out, double* const* z_out,
                        scuc_solve_info* infos, scuc_batch_info* binfo);

/* ---------------------------------------------------------------------- */
/* Transmission filtering (Fig. 1): the LP is solved without the network    */
/* security rows; the rows of a pool that the solution violates are added   */
/* and the LP is re-solved from the previous point, until none is violated. */
/* ---------------------------------------------------------------------- */
/* Rows of the pool LP (its rows, same columns as the LP being filtered)
 * violated at x: lo_i - a_i x > tol (1 + |lo_i|) or a_i x - hi_i > tol (1 +
 * |hi_i|) over the finite bounds (a_i x in FP64, unscaled values).
 *  x[n]: host (x_on_device = 0) or device pointer on the pool's device.
 *  rows_out[cap]: receives the first min(count, cap) violated row indices
 *    in increasing order (host); *count_out the number violated (may exceed
 *    cap); *worst_out (may be NULL) the largest relative violation, 0 when
 *    none.  SCUC_E_INVALID for a null handle or x, cap < 0, tol < 0.  */
int scuc_lp_row_violations(scuc_lp* pool, const double* x, int32_t x_on_device, double tol, int32_t* rows_out,
                           int32_t cap, int32_t* count_out, double* worst_out);

/* A new LP with base's rows followed by the pool rows rows[count] (in that
 * order, host array, repeats allowed); costs and column bounds are base's
 * current ones.  Built on the device from device copies; *out is a new
 * handle on base's stream (caller destroys it).  SCUC_E_INVALID when the
 * pool has another column count or device, or a row is out of range
 * (nothing is created).                                                  */
int scuc_lp_add_rows(scuc_lp* base, scuc_lp* pool, const int32_t* rows, int32_t count, scuc_lp** out);

/* ---------------------------------------------------------------------- */
/* Logic-driven fixing and presolve (Sec. 4.1 Round + Algorithm 1; the      */
/* MILP-/LP-Presolve steps of Algorithm 2, Sec. 4.2)                        */
/* ---------------------------------------------------------------------- */
typedef struct {
  int32_t G, T;            /* generators, hours                              */
  const int32_t* u_idx;    /* [G*T] column of u_{g,t}, index g*T + t (host)  */
  const int32_t* v_idx;    /* [G*T] column of v_{g,t}                        */
  const int32_t* w_idx;    /* [G*T] column of w_{g,t}                        */
  const int8_t* u_init;    /* [G] commitment before the first hour (0/1)     */
} scuc_map;

typedef struct {
  double tau;              /* Round threshold, 0 <= tau < 0.5 (0.1)          */
  int32_t t_first;         /* 1: Algorithm 1 from the second hour (as
                              written); 0: also the first, against u_init   */
  int32_t max_passes;      /* propagation passes (100)                       */
  int32_t x_on_device;     /* x_relaxed is a device pointer (0)              */
  int32_t build_reduced;   /* build the reduced LP when asked for (1)        */
} scuc_fix_params;

typedef struct {
  int64_t nfixed;          /* (g,t) triples fixed by Algorithm 1             */
  int32_t passes;          /* propagation passes run                         */
  int32_t infeasible;      /* bounds crossed, or an emptied row is violated  */
  int32_t m_red, n_red;    /* reduced LP size                                */
  int64_t nnz_red;
  int64_t n_fixed_cols;    /* columns with xl == xu after propagation        */
  double obj_const;        /* c^T x of the removed (fixed) columns           */
  double ms;               /* wall time of the call                          */
  double ms_propagate;     /* of which Round, Algorithm 1 and propagation     */
  double ms_reduce;        /* ... the reduced CSR and maps                    */
  double ms_setup;         /* ... the reduced LP's device setup (transpose,
                              partitions, buffers)                          */
} scuc_fix_info;

void scuc_default_fix_params(scuc_fix_params* p);

/* One fixing round on the model held by lp (the relaxed MILP M):
 *  1. Round(x, tau) of every u, v, w value of x_relaxed[n] (unscaled, host
 *     or device per p->x_on_device) and Algorithm 1 per generator: hours are
 *     fixed in order while all four rounded values are confident and
 *     u_t - u_{t-1} = v_t - w_t, v_t + w_t <= 1 (Eq. 1); fix_out[3*(g*T+t)
 *     + {0,1,2}] (host, nullable) = fixed u, v, w or -1.
 *  2. The fixed columns get xl = xu = value in lp's bounds (M is updated).
 *  3. Bound propagation (Jacobi passes until no change or max_passes):
 *     each row's activity range bounds every column of the row; integer
 *     columns (is_int[n], host, nullable = the map's u, v, w) are rounded
 *     inward with 1e-6 slack; continuous changes below 1e-9 relative are
 *     ignored.  lp's bounds receive the result.
 *  4. Reduced LP: fixed columns removed and folded into the row bounds,
 *     rows whose activity range lies inside [lo, hi] removed.
 *     *reduced_out (nullable) receives a new handle (caller destroys) on the
 *     caller's stream of lp; col_map_out[n_red] / row_map_out[m_red] (host,
 *     nullable, sized n / m) map reduced indices to lp's indices.
 * Returns SCUC_E_INFEASIBLE (info->infeasible = 1) when propagation crosses
 * a column's bounds or an emptied row is violated; no reduced LP then.   */
int scuc_fix_and_propagate(scuc_lp* lp, const scuc_map* map, const uint8_t* is_int,
                           const double* x_relaxed, const scuc_fix_params* p, int8_t* fix_out,
                           scuc_lp** reduced_out, int32_t* col_map_out, int32_t* row_map_out,
                           scuc_fix_info* info);

/* Host copies of the handle's column bounds (xl, xu nullable, length n). */
int scuc_lp_get_bounds(const scuc_lp* lp, double* xl, double* xu);

/* Replace the handle's column bounds (n each): host arrays (validated: no
 * NaN, xl <= xu, xl != +INF, xu != -INF) or, with on_device = 1, device
 * arrays on the handle's device (not validated).  Used to restore or set
 * the bounds of the model between fixing rounds.                        */
int scuc_lp_set_bounds(scuc_lp* lp, const double* xl, const double* xu, int32_t on_device);

/* Host copies of the handle's LP (each pointer nullable): row_ptr[m+1],
 * col[nnz], val[nnz], c[n], xl[n], xu[n], lo[m], hi[m] (unscaled).      */
int scuc_lp_export(const scuc_lp* lp, int64_t* row_ptr, int32_t* col, double* val, double* c,
                   double* xl, double* xu, double* lo, double* hi);

/* KKT residuals of a caller-supplied point, with no device allocation.
 * The paper has no counterpart; this is a service for callers that cannot
 * allocate GPU memory at the point of the call: code whose device memory is
 * already handed out to another allocator or a fixed pool, or a serving loop
 * that must not pay for cudaMalloc/cudaFree (cudaFree waits for the whole
 * device).  The handle itself is created beforehand as usual.
 *  x_dev[n], y_dev[m], z_dev[n]: device pointers on the handle's device
 *    (unscaled point; z is used as given).  out_dev[6]: device pointer that
 *    receives {r_p, r_d, gap, pobj, dobj, kkt}, the same quantities that
 *    scuc_lp_solve reports for its returned point.
 *  Work is queued on the handle's stream order; the call does not wait for
 *    it, so synchronise the creation stream before reading out_dev.
 *  The partial sums go to one fixed device array of 2^20 doubles (8 MiB),
 *    which every GPU that loads this library holds until the process exits.
 *    An LP that needs more slots (3 per row block of A plus 4 per row block
 *    of A^T) is rejected with SCUC_E_INVALID and a message naming the sizes.
 *  The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and keeps it for the device's current context;
 *    make that first call before any stream capture on that device.  After
 *    a device reset the next call (with a new handle) looks it up again.
 *  kkt is the largest of r_p, r_d and gap, or NaN when one of them is NaN.
 *  All calls share the one array: calls whose work overlaps on the GPU (for
 *    example on two unsynchronised streams) race on it.  Each call writes
 *    every slot it later reads, so contents left by earlier calls are never
 *    used.                                                               */
int scuc_lp_kkt_noalloc(scuc_lp* lp, const double* x_dev, const double* y_dev, const double* z_dev,
                        double* out_dev);

/* FMA throughput of the current device, measured (no counterpart in the
 * paper): every thread of 8 blocks per SM runs eight independent
 * register-resident FMA chains of 16,384 steps; the best of three timed
 * launches after one warm-up (CUDA events), clocks left as they are.
 * fp64: 1 for FP64 (DFMA), 0 for FP32.  tflops receives 2 * FMAs / time in
 * TFLOP/s, ms (nullable) the launch time.  The FP64 SpMV kernels are bound
 * by this rate as much as by HBM (one DFMA per nonzero).  Allocates and
 * frees a small device buffer; SCUC_E_CUDA on a CUDA error.            */
int scuc_probe_fma_peak(int32_t fp64, double* tflops, double* ms);

void scuc_lp_destroy(scuc_lp* lp);

const char* scuc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
