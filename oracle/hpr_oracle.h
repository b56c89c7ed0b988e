/*
 * Plain FP64 CPU oracle for the restarted HPR LP solve (Sec. 3, Eq. 9), the
 * Round operator and Algorithm 1 (Sec. 4.1), and the bound-propagation
 * presolve that stands in for MILP-/LP-Presolve of Algorithm 2 (Sec. 4.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the CUDA library includes, links or
 * calls this code; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It is deliberately scalar and unblocked so that
 * each loop can be read against the paper.
 */
#ifndef HPR_ORACLE_H
#define HPR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* LP  min c^T x  s.t.  lo <= A x <= hi,  xl <= x <= xu   (Eq. 8 with the row
 * set generalised from {Ax >= theta} to a box; +-INFINITY allowed).        */
typedef struct {
  int32_t m, n;
  const int64_t* row_ptr; /* [m+1] */
  const int32_t* col;     /* [nnz] */
  const double* val;      /* [nnz] */
  const double* c;        /* [n] */
  const double* xl;       /* [n] */
  const double* xu;       /* [n] */
  const double* lo;       /* [m] */
  const double* hi;       /* [m] */
} orc_lp;

typedef struct {
  double tol;            /* stop when max(r_p, r_d, gap) <= tol            */
  int64_t max_iter;
  int32_t check_every;   /* KKT / restart evaluation period               */
  int32_t use_scaling;   /* 1: Pock-Chambolle + normalisation (Sec. 3.A);
                            2: Ruiz (10 passes) first, then as 1; 0: none */
  double sigma0;         /* initial primal step                           */
  double lambda_in;      /* > 0: use this lambda instead of power method  */
  double lambda_safety;  /* lambda = safety * power-method estimate       */
  int32_t power_max_iter;
  double power_tol;
  uint64_t power_seed;   /* start vector: SplitMix64(seed + (j+1)*golden) */
  double restart_suff;   /* 0.2 */
  double restart_nec;    /* 0.8 */
  double restart_long;   /* 0.2 */
  int32_t log_cap;       /* capacity of the check log                     */
  int32_t restart_ref;   /* reference rho0 of the restart tests: 0 = metric
                            at the first check of the cycle, 1 = metric at
                            the check that made the last restart           */
  int32_t restart_metric;/* 0: rho^2 = ||dx||^2/sigma + lambda sigma ||dy||^2;
                            1: the same plus the cross term 2<A dx, dy> (the
                            norm in which the iteration is nonexpansive);
                            2: the KKT error max(r_p, r_d, gap)            */
  int32_t sigma_update;  /* 1: sigma update at restarts; 0: keep sigma0    */
  int32_t algo;          /* 0: restarted HPR (Eq. 9, Halpern step);
                            1: restarted PDHG with ergodic averaging: the
                            same two steps, no Halpern step, checks and
                            restarts on the running average of the cycle  */
  double infeas_tol;     /* > 0: infeasibility detection at every check
                            (relative violation of the certificate)       */
} orc_params;

typedef struct {
  int64_t iter;      /* total iterations when the check was taken   */
  int32_t restart;   /* 1 if this check restarted the cycle         */
  int32_t first;     /* 1 if first check of its cycle                */
  double rp, rd, gap, pobj, dobj, rho, sigma;
  double rmap;       /* ||R(x_bar, y_bar, z_bar)|| of Theorem 1, unscaled */
} orc_log;

typedef struct {
  int64_t iters;
  int32_t status;    /* 0 optimal, 1 iteration limit, 3 numerical (a
                        residual is NaN or infinite), 5 primal
                        infeasible, 6 dual infeasible (primal unbounded) */
  int32_t restarts;
  int32_t nlog;
  int32_t power_iters;
  double kkt, rp, rd, gap, pobj, dobj, lambda, sigma, beta, gamma;
} orc_info;

/* Sec. 3.A last paragraph: Pock-Chambolle (alpha = 1) diagonal scaling and
 * normalisation of the bound and cost vectors.  Outputs the scaled data.  */
void orc_scale(const orc_lp* lp, int32_t use_scaling, double* Dr, double* Dc, double* beta,
               double* gamma, double* val_s, double* c_s, double* xl_s, double* xu_s,
               double* lo_s, double* hi_s);

/* Power method for lambda_max(A A^T) (Sec. 3, text after Eq. 9). */
double orc_power_lambda(int32_t m, int32_t n, const int64_t* rp, const int32_t* col,
                        const double* val, int32_t max_iter, double tol, uint64_t seed,
                        int32_t* iters_out);

/* Restarted HPR iteration (Eq. 9), or restarted PDHG with ergodic averaging
 * (algo = 1).  x_init / y_init may be NULL.  With status 5 y_out holds the
 * dual ray that certifies primal infeasibility, with status 6 x_out holds
 * the primal ray that certifies unboundedness (both unscaled). */
int orc_hpr_solve(const orc_lp* lp, const orc_params* prm, const double* x_init,
                  const double* y_init, double* x_out, double* y_out, double* z_out,
                  orc_info* info, orc_log* log);

/* KKT residuals of (x, y, z) on the unscaled LP: out = {rp, rd, gap, pobj,
 * dobj, kkt, ||R||} (out holds 7).  z is used as given (the caller
 * projects it).                                                          */
void orc_kkt(const orc_lp* lp, const double* x, const double* y, const double* z, double* out);

/* Threads of the OpenMP build (k > 0 sets them); returns the threads that
 * loops will use (1 in the single-threaded build).                       */
int32_t orc_set_threads(int32_t k);

/* Round(s, tau) (Sec. 4.1). */
int32_t orc_round(double s, double tau);

/* Algorithm 1.  u, v, w: relaxed values indexed g*T + t.  fix_out[3*(g*T+t)
 * + {0,1,2}] = 0/1 fixed value of (u, v, w), or -1 when left free.
 * t_first = 1 is the literal reading (hour 1 never fixed); t_first = 0 also
 * tests hour 1 against u_init.  Returns the number of fixed (g,t) triples. */
int64_t orc_fix(int32_t G, int32_t T, const double* u, const double* v, const double* w,
                const int8_t* u_init, double tau, int32_t t_first, int8_t* fix_out);

/* Jacobi activity-based bound propagation on  lo <= A x <= hi.  xl/xu are
 * updated in place.  Returns passes used, or -1 - pass when a column's
 * bounds cross (infeasible).                                              */
int32_t orc_propagate(int32_t m, int32_t n, const int64_t* rp, const int32_t* col,
                      const double* val, const double* lo, const double* hi, double* xl,
                      double* xu, const uint8_t* is_int, int32_t max_passes);

/* Removal of fixed columns (folded into the row bounds) and of rows whose
 * activity range lies inside [lo, hi].  Sizes of the reduced LP returned in
 * dims = {m_r, n_r, nnz_r}; output arrays must hold the unreduced sizes.
 * Returns 0, or 1 when an emptied row is violated.                        */
int orc_reduce(int32_t m, int32_t n, const int64_t* rp, const int32_t* col, const double* val,
               const double* c, const double* lo, const double* hi, const double* xl,
               const double* xu, int64_t* dims, int64_t* rp_r, int32_t* col_r, double* val_r,
               double* c_r, double* lo_r, double* hi_r, double* xl_r, double* xu_r,
               int32_t* row_map, int32_t* col_map, double* obj_const);

#ifdef __cplusplus
}
#endif
#endif
