/*
 * Plain FP64 CPU oracle: restarted HPR for LP (Sec. 3, Eq. 9 and Theorem 1),
 * Pock-Chambolle scaling with normalisation (Sec. 3.A), the Round operator
 * and Algorithm 1 (Sec. 4.1), and the bound propagation + reduction that
 * stands in for MILP-/LP-Presolve in Algorithm 2 (Sec. 4.2).
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).  It shares no
 * source with the CUDA library.  Every loop is scalar, sequential and in the
 * order the formulas are written; no blocking, fusion or reordering.
 *
 * Points the paper leaves open (restart rule, sigma update, residual
 * normalisation, propagation tolerances) are settled by a stated reading,
 * each written out where it is used below.  Every sum runs over its terms in
 * index order.
 */
#include "hpr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* The same source builds single-threaded (the oracle the tests use) and with
 * OpenMP (a timing baseline on all host cores): the pragmas only split
 * loops whose iterations are independent, and every row or column sum keeps
 * its order.  Only the scalar sums marked "reduction" (norms, dot products)
 * are added in a different order when more than one thread runs.         */
#define ORC_STR(x) #x
#ifdef _OPENMP
#define ORC_PAR(clauses) _Pragma(ORC_STR(omp parallel for schedule(static) clauses))
#define ORC_PAR_ROWS _Pragma("omp parallel for schedule(dynamic, 256)")
#else
#define ORC_PAR(clauses)
#define ORC_PAR_ROWS
#endif

int32_t orc_set_threads(int32_t k) {
#ifdef _OPENMP
  if (k > 0) omp_set_num_threads(k);
  return (int32_t)omp_get_max_threads();
#else
  (void)k;
  return 1;
#endif
}

static double clampd(double v, double l, double u) {
  if (v < l) return l;
  if (v > u) return u;
  return v;
}

/* magnitude of the finite bounds of one row (0 when both are infinite) */
static double bound_mag(double lo, double hi) {
  double b = 0.0;
  if (isfinite(lo) && fabs(lo) > b) b = fabs(lo);
  if (isfinite(hi) && fabs(hi) > b) b = fabs(hi);
  return b;
}

static double* dalloc(int64_t k) { return (double*)calloc((size_t)(k > 0 ? k : 1), sizeof(double)); }

/* y = A x (CSR): y_i = sum_k a_ik x_k over the row's entries in order */
static void spmv(int32_t m, const int64_t* rp, const int32_t* col, const double* val,
                 const double* x, double* y) {
  ORC_PAR_ROWS
  for (int32_t i = 0; i < m; i++) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; k++) s += val[k] * x[col[k]];
    y[i] = s;
  }
}

/* Column index of a CSR matrix: the entries of column j, in increasing row
 * order, are the CSR positions pos[cp[j] .. cp[j+1]) of rows row[...].    */
typedef struct {
  int64_t* cp;
  int32_t* row;
  int64_t* pos;
} orc_cols;

static void cols_build(int32_t m, int32_t n, const int64_t* rp, const int32_t* col, orc_cols* t) {
  const int64_t nnz = rp[m];
  t->cp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  t->row = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  t->pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  for (int64_t k = 0; k < nnz; k++) t->cp[col[k] + 1]++;
  for (int32_t j = 0; j < n; j++) t->cp[j + 1] += t->cp[j];
  int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t j = 0; j < n; j++) next[j] = t->cp[j];
  for (int32_t i = 0; i < m; i++)
    for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
      const int64_t p = next[col[k]]++;
      t->row[p] = i;
      t->pos[p] = k;
    }
  free(next);
}

static void cols_free(orc_cols* t) {
  free(t->cp);
  free(t->row);
  free(t->pos);
}

/* y = A^T x: y_j = sum_i a_ij x_i over the column's entries in row order */
static void spmv_t(int32_t n, const orc_cols* t, const double* val, const double* x, double* y) {
  ORC_PAR_ROWS
  for (int32_t j = 0; j < n; j++) {
    double s = 0.0;
    for (int64_t p = t->cp[j]; p < t->cp[j + 1]; p++) s += val[t->pos[p]] * x[t->row[p]];
    y[j] = s;
  }
}

static double dot(int64_t k, const double* a, const double* b) {
  double s = 0.0;
  ORC_PAR(reduction(+ : s))
  for (int64_t i = 0; i < k; i++) s += a[i] * b[i];
  return s;
}

/* ---------------------------------------------------------------------- */
/* Sec. 3.A: Pock-Chambolle scaling (alpha = 1) and normalisation          */
/* ---------------------------------------------------------------------- */
void orc_scale(const orc_lp* lp, int32_t use_scaling, double* Dr, double* Dc, double* beta,
               double* gamma, double* val_s, double* c_s, double* xl_s, double* xu_s,
               double* lo_s, double* hi_s) {
  const int32_t m = lp->m, n = lp->n;
  for (int32_t i = 0; i < m; i++) Dr[i] = 1.0;
  for (int32_t j = 0; j < n; j++) Dc[j] = 1.0;
  double* rs = dalloc(m);
  double* cs = dalloc(n);
  if (use_scaling == 2) {
    /* Ruiz: 10 passes; each divides every row and column of the current
     * D_r A D_c by the square root of its largest magnitude */
    for (int pass = 0; pass < 10; pass++) {
      for (int32_t i = 0; i < m; i++) rs[i] = 0.0;
      for (int32_t j = 0; j < n; j++) cs[j] = 0.0;
      for (int32_t i = 0; i < m; i++)
        for (int64_t k = lp->row_ptr[i]; k < lp->row_ptr[i + 1]; k++) {
          const double a = fabs((Dr[i] * lp->val[k]) * Dc[lp->col[k]]);
          if (a > rs[i]) rs[i] = a;
          if (a > cs[lp->col[k]]) cs[lp->col[k]] = a;
        }
      for (int32_t i = 0; i < m; i++) Dr[i] *= rs[i] > 0.0 ? 1.0 / sqrt(rs[i]) : 1.0;
      for (int32_t j = 0; j < n; j++) Dc[j] *= cs[j] > 0.0 ? 1.0 / sqrt(cs[j]) : 1.0;
    }
  }
  if (use_scaling >= 1) {
    /* Pock-Chambolle (alpha = 1) on the current matrix:
     * D_r,i *= 1/sqrt(sum_j |a_ij|),  D_c,j *= 1/sqrt(sum_i |a_ij|) */
    for (int32_t j = 0; j < n; j++) cs[j] = 0.0;
    for (int32_t i = 0; i < m; i++) {
      double s = 0.0;
      for (int64_t k = lp->row_ptr[i]; k < lp->row_ptr[i + 1]; k++) {
        const double a = fabs((Dr[i] * lp->val[k]) * Dc[lp->col[k]]);
        s += a;
        cs[lp->col[k]] += a;
      }
      rs[i] = s;
    }
    for (int32_t i = 0; i < m; i++) Dr[i] *= rs[i] > 0.0 ? 1.0 / sqrt(rs[i]) : 1.0;
    for (int32_t j = 0; j < n; j++) Dc[j] *= cs[j] > 0.0 ? 1.0 / sqrt(cs[j]) : 1.0;
  }
  free(rs);
  free(cs);
  /* A_hat = D_r A D_c; bounds and cost in the scaled variables x = D_c x_hat */
  for (int32_t i = 0; i < m; i++)
    for (int64_t k = lp->row_ptr[i]; k < lp->row_ptr[i + 1]; k++)
      val_s[k] = (Dr[i] * lp->val[k]) * Dc[lp->col[k]];
  for (int32_t j = 0; j < n; j++) {
    c_s[j] = Dc[j] * lp->c[j];
    xl_s[j] = lp->xl[j] / Dc[j];
    xu_s[j] = lp->xu[j] / Dc[j];
  }
  for (int32_t i = 0; i < m; i++) {
    lo_s[i] = Dr[i] * lp->lo[i];
    hi_s[i] = Dr[i] * lp->hi[i];
  }
  /* normalisation of the bound vector by 1+||b|| and the cost by 1+||c|| */
  double bn = 0.0, cn = 0.0;
  for (int32_t i = 0; i < m; i++) {
    double b = bound_mag(lo_s[i], hi_s[i]);
    bn += b * b;
  }
  for (int32_t j = 0; j < n; j++) cn += c_s[j] * c_s[j];
  *beta = use_scaling ? 1.0 + sqrt(bn) : 1.0;
  *gamma = use_scaling ? 1.0 + sqrt(cn) : 1.0;
  for (int32_t i = 0; i < m; i++) {
    lo_s[i] /= *beta;
    hi_s[i] /= *beta;
  }
  for (int32_t j = 0; j < n; j++) {
    xl_s[j] /= *beta;
    xu_s[j] /= *beta;
    c_s[j] /= *gamma;
  }
}

/* ---------------------------------------------------------------------- */
/* Power method for lambda_max(A A^T) (Sec. 3)                             */
/* ---------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea, Flood 2014) evaluated at counter j */
static uint64_t splitmix64_at(uint64_t seed, uint64_t j) {
  uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static double power_lambda(int32_t m, int32_t n, const int64_t* rp, const int32_t* col,
                           const orc_cols* tc, const double* val, int32_t max_iter, double tol,
                           uint64_t seed, int32_t* iters_out) {
  double* q = dalloc(n);
  double* u = dalloc(m);
  double* w = dalloc(n);
  for (int32_t j = 0; j < n; j++) q[j] = 0.5 + (double)(splitmix64_at(seed, (uint64_t)j) >> 11) * 0x1.0p-53;
  double nq = sqrt(dot(n, q, q));
  ORC_PAR()
  for (int32_t j = 0; j < n; j++) q[j] /= nq;
  double lam = 0.0, lam_prev = 0.0;
  int32_t it = 0;
  for (it = 1; it <= max_iter; it++) {
    spmv(m, rp, col, val, q, u);           /* u = A q          */
    spmv_t(n, tc, val, u, w);              /* w = A^T A q      */
    lam = dot(m, u, u);                    /* q^T A^T A q      */
    double nw = sqrt(dot(n, w, w));
    if (nw == 0.0) break;
    ORC_PAR()
    for (int32_t j = 0; j < n; j++) q[j] = w[j] / nw;
    if (it > 1 && fabs(lam - lam_prev) <= tol * lam) break;
    lam_prev = lam;
  }
  if (it > max_iter) it = max_iter;
  if (iters_out) *iters_out = it;
  free(q);
  free(u);
  free(w);
  return lam;
}

double orc_power_lambda(int32_t m, int32_t n, const int64_t* rp, const int32_t* col,
                        const double* val, int32_t max_iter, double tol, uint64_t seed,
                        int32_t* iters_out) {
  orc_cols tc;
  cols_build(m, n, rp, col, &tc);
  double lam = power_lambda(m, n, rp, col, &tc, val, max_iter, tol, seed, iters_out);
  cols_free(&tc);
  return lam;
}

/* ---------------------------------------------------------------------- */
/* KKT residuals on the unscaled LP (Theorem 1 map, normalised)            */
/* ---------------------------------------------------------------------- */
static void kkt(const orc_lp* lp, const orc_cols* tc, const double* x, const double* y,
                const double* z, double* out) {
  const int32_t m = lp->m, n = lp->n;
  double* ax = dalloc(m);
  double* aty = dalloc(n);
  spmv(m, lp->row_ptr, lp->col, lp->val, x, ax);
  spmv_t(n, tc, lp->val, y, aty);
  /* primal: distance of A x to [lo, hi] */
  double pr = 0.0, bn = 0.0;
  ORC_PAR(reduction(+ : pr, bn))
  for (int32_t i = 0; i < m; i++) {
    double d = ax[i] - clampd(ax[i], lp->lo[i], lp->hi[i]);
    pr += d * d;
    double b = bound_mag(lp->lo[i], lp->hi[i]);
    bn += b * b;
  }
  /* dual: c - A^T y - z */
  double dr = 0.0, cn = 0.0;
  ORC_PAR(reduction(+ : dr, cn))
  for (int32_t j = 0; j < n; j++) {
    double d = lp->c[j] - aty[j] - z[j];
    dr += d * d;
    cn += lp->c[j] * lp->c[j];
  }
  /* objectives: dual uses the bound each multiplier prices */
  double pobj = 0.0, dobj = 0.0;
  ORC_PAR(reduction(+ : pobj))
  for (int32_t j = 0; j < n; j++) pobj += lp->c[j] * x[j];
  ORC_PAR(reduction(+ : dobj))
  for (int32_t i = 0; i < m; i++) {
    if (y[i] > 0.0 && isfinite(lp->lo[i])) dobj += lp->lo[i] * y[i];
    else if (y[i] < 0.0 && isfinite(lp->hi[i])) dobj += lp->hi[i] * y[i];
  }
  ORC_PAR(reduction(+ : dobj))
  for (int32_t j = 0; j < n; j++) {
    if (z[j] > 0.0 && isfinite(lp->xl[j])) dobj += lp->xl[j] * z[j];
    else if (z[j] < 0.0 && isfinite(lp->xu[j])) dobj += lp->xu[j] * z[j];
  }
  out[0] = sqrt(pr) / (1.0 + sqrt(bn));
  out[1] = sqrt(dr) / (1.0 + sqrt(cn));
  out[2] = fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
  out[3] = pobj;
  out[4] = dobj;
  /* the largest of the three; NaN if any of them is NaN */
  out[5] = (isnan(out[0]) || isnan(out[1]) || isnan(out[2])) ? NAN : fmax(out[0], fmax(out[1], out[2]));
  /* Theorem 1 map R(x,y,z) with the row box generalising R^m_+:
   * R1 = y - P(y - A x), P(r) = r + Pi_[lo,hi](-r)  (= Pi_+(y - Ax + theta)
   * for rows A x >= theta);  R2 = x - Pi_K(x - z);  R3 = c - A^T y - z   */
  double rr = 0.0;
  ORC_PAR(reduction(+ : rr))
  for (int32_t i = 0; i < m; i++) {
    double r = y[i] - ax[i];
    double p = r + clampd(-r, lp->lo[i], lp->hi[i]);
    rr += (y[i] - p) * (y[i] - p);
  }
  ORC_PAR(reduction(+ : rr))
  for (int32_t j = 0; j < n; j++) {
    double r2 = x[j] - clampd(x[j] - z[j], lp->xl[j], lp->xu[j]);
    double r3 = lp->c[j] - aty[j] - z[j];
    rr += r2 * r2 + r3 * r3;
  }
  out[6] = sqrt(rr);
  free(ax);
  free(aty);
}

void orc_kkt(const orc_lp* lp, const double* x, const double* y, const double* z, double* out) {
  orc_cols tc;
  cols_build(lp->m, lp->n, lp->row_ptr, lp->col, &tc);
  kkt(lp, &tc, x, y, z, out);
  cols_free(&tc);
}

/* ---------------------------------------------------------------------- */
/* Infeasibility certificates on the scaled LP (an LP of the same form:     */
/* scaling maps certificates to certificates).  The paper defines no        */
/* infeasibility test; these are the Farkas and recession-cone certificates */
/* of LP duality for Eq. 8 with a row box, tested on the step displacement  */
/* (for an infeasible LP it tends to the iteration's minimal displacement). */
/* ---------------------------------------------------------------------- */
/* Primal infeasibility (Farkas): a dual ray u with z = -A^T u has the
 * homogeneous dual objective  sum_i (u_i > 0 ? lo_i : hi_i) u_i
 * + sum_j (z_j > 0 ? xl_j : xu_j) z_j  > 0.  Terms that would need an
 * infinite bound are not summed; their squares make up the violation.
 * The ray is accepted when the objective F > 0 and ||violation|| <= tol F. */
static int primal_infeasible(int32_t m, int32_t n, const orc_cols* tc, const double* val,
                             const double* lo, const double* hi, const double* xl,
                             const double* xu, const double* u, double tol) {
  double* aty = dalloc(n);
  spmv_t(n, tc, val, u, aty);
  double F = 0.0, V = 0.0;
  for (int32_t i = 0; i < m; i++) {
    if (u[i] > 0.0) {
      if (isfinite(lo[i])) F += lo[i] * u[i];
      else V += u[i] * u[i];
    } else if (u[i] < 0.0) {
      if (isfinite(hi[i])) F += hi[i] * u[i];
      else V += u[i] * u[i];
    }
  }
  for (int32_t j = 0; j < n; j++) {
    const double z = -aty[j];
    if (z > 0.0) {
      if (isfinite(xl[j])) F += xl[j] * z;
      else V += z * z;
    } else if (z < 0.0) {
      if (isfinite(xu[j])) F += xu[j] * z;
      else V += z * z;
    }
  }
  free(aty);
  return F > 0.0 && sqrt(V) <= tol * F;
}

/* Dual infeasibility (primal unbounded): a direction d with c^T d < 0 that
 * stays in the recession cones, A d in that of [lo, hi] ((A d)_i >= 0 where
 * lo_i is finite, <= 0 where hi_i is finite) and d in that of [xl, xu].
 * Accepted when c^T d < 0 and ||cone violation|| <= tol |c^T d|.          */
static int dual_infeasible(int32_t m, int32_t n, const int64_t* rp, const int32_t* col,
                           const double* val, const double* c, const double* lo, const double* hi,
                           const double* xl, const double* xu, const double* d, double tol) {
  double* ad = dalloc(m);
  spmv(m, rp, col, val, d, ad);
  double cd = 0.0, V = 0.0;
  for (int32_t j = 0; j < n; j++) {
    cd += c[j] * d[j];
    if (d[j] < 0.0 && isfinite(xl[j])) V += d[j] * d[j];
    if (d[j] > 0.0 && isfinite(xu[j])) V += d[j] * d[j];
  }
  for (int32_t i = 0; i < m; i++) {
    if (ad[i] < 0.0 && isfinite(lo[i])) V += ad[i] * ad[i];
    if (ad[i] > 0.0 && isfinite(hi[i])) V += ad[i] * ad[i];
  }
  free(ad);
  return cd < 0.0 && sqrt(V) <= tol * (-cd);
}

/* ---------------------------------------------------------------------- */
/* Restarted HPR (Eq. 9); restarted PDHG with ergodic averaging (algo 1)   */
/* ---------------------------------------------------------------------- */
int orc_hpr_solve(const orc_lp* lp, const orc_params* prm, const double* x_init,
                  const double* y_init, double* x_out, double* y_out, double* z_out,
                  orc_info* info, orc_log* log) {
  const int32_t m = lp->m, n = lp->n;
  const int64_t nnz = lp->row_ptr[m];
  double *Dr = dalloc(m), *Dc = dalloc(n), *vs = dalloc(nnz), *cs = dalloc(n);
  double *xls = dalloc(n), *xus = dalloc(n), *los = dalloc(m), *his = dalloc(m);
  double beta = 1.0, gamma = 1.0;
  orc_scale(lp, prm->use_scaling, Dr, Dc, &beta, &gamma, vs, cs, xls, xus, los, his);
  orc_cols tc; /* A^T products run over the columns, each in row order */
  cols_build(m, n, lp->row_ptr, lp->col, &tc);

  double lambda = prm->lambda_in;
  int32_t piters = 0;
  if (!(lambda > 0.0)) {
    lambda = prm->lambda_safety *
             power_lambda(m, n, lp->row_ptr, lp->col, &tc, vs, prm->power_max_iter, prm->power_tol,
                          prm->power_seed, &piters);
    if (!(lambda > 0.0)) lambda = 1.0; /* no constraints: any positive value */
  }

  double *x = dalloc(n), *x0 = dalloc(n), *xt = dalloc(n), *xb = dalloc(n), *zb = dalloc(n);
  double *g = dalloc(n), *y = dalloc(m), *y0 = dalloc(m), *yb = dalloc(m), *q = dalloc(m);
  double *xo = dalloc(n), *yo = dalloc(m), *zo = dalloc(n);
  double *dyv = dalloc(m), *pv = dalloc(m);
  /* PDHG: the step's x_bar, the running averages of the cycle, and the ray
   * x_bar - x of a check iteration */
  const int pdhg = prm->algo == 1;
  double *xbr = dalloc(n), *xavg = dalloc(n), *yavg = dalloc(m), *dxv = dalloc(n);

  /* starting point, in scaled variables, projected onto K and the dual cone */
  ORC_PAR()
  for (int32_t j = 0; j < n; j++) {
    double v = x_init ? x_init[j] / (beta * Dc[j]) : 0.0;
    x[j] = clampd(v, xls[j], xus[j]);
  }
  ORC_PAR()
  for (int32_t i = 0; i < m; i++) {
    double v = y_init ? y_init[i] / (gamma * Dr[i]) : 0.0;
    if (!isfinite(los[i]) && v > 0.0) v = 0.0;
    if (!isfinite(his[i]) && v < 0.0) v = 0.0;
    y[i] = v;
  }
  memcpy(x0, x, sizeof(double) * (size_t)n);
  memcpy(y0, y, sizeof(double) * (size_t)m);

  double sigma = prm->sigma0;
  int64_t k = 0, t = 0;
  int first_check = 1;
  double rho0 = 0.0, rho_prev = 0.0;
  int32_t restarts = 0, nlog = 0, status = 1;
  double last[7] = {0, 0, 0, 0, 0, 0, 0};
  int have_out = 0;

  while (t < prm->max_iter) {
    const int is_check = ((t + 1) % prm->check_every == 0) || (t + 1 == prm->max_iter);
    const double s = 1.0 / (lambda * sigma);
    /* HPR: Halpern weights; PDHG: weights of the running average */
    const double wa = pdhg ? 1.0 / (double)(k + 1) : 1.0 / (double)(k + 2);
    const double wb = pdhg ? (double)k / (double)(k + 1) : (double)(k + 1) / (double)(k + 2);

    /* x_bar = Pi_K(x + sigma (A^T y - c)); z_bar = (x_bar - v)/sigma */
    spmv_t(n, &tc, vs, y, g);
    double dxx = 0.0;
    ORC_PAR(reduction(+ : dxx))
    for (int32_t j = 0; j < n; j++) {
      double v = x[j] + sigma * (g[j] - cs[j]);
      double xbar = clampd(v, xls[j], xus[j]);
      xt[j] = 2.0 * xbar - x[j];                   /* reflection */
      if (pdhg) {
        xbr[j] = xbar;
        xavg[j] = wa * xbar + wb * xavg[j];
      }
      if (is_check) {
        xb[j] = pdhg ? xavg[j] : xbar;
        zb[j] = (xbar - v) / sigma;                /* PDHG: replaced below */
        dxv[j] = xbar - x[j];
        dxx += (xbar - x[j]) * (xbar - x[j]);
      }
    }
    /* y_bar = prox: r = y - s A x_tilde; y_bar = r + s * Pi_[lo,hi](-r/s) */
    spmv(m, lp->row_ptr, lp->col, vs, xt, q);
    double dyy = 0.0;
    ORC_PAR(reduction(+ : dyy))
    for (int32_t i = 0; i < m; i++) {
      double r = y[i] - s * q[i];
      double ybar = r + s * clampd(-r / s, los[i], his[i]);
      if (pdhg) yavg[i] = wa * ybar + wb * yavg[i];
      if (is_check) {
        yb[i] = pdhg ? yavg[i] : ybar;
        dyv[i] = ybar - y[i];
        dyy += (ybar - y[i]) * (ybar - y[i]);
      }
      if (pdhg) y[i] = ybar;                         /* PDHG step */
      else y[i] = wa * y0[i] + wb * (2.0 * ybar - y[i]);  /* Halpern step */
    }
    ORC_PAR()
    for (int32_t j = 0; j < n; j++) x[j] = pdhg ? xbr[j] : wa * x0[j] + wb * xt[j];
    k++;
    t++;
    if (!is_check) continue;

    /* PDHG: the checked point is the average; its z is the reduced cost
     * c - A^T y_avg where the bounds let it act, 0 elsewhere (the scaled
     * copy is zeroed below where a bound is infinite) */
    if (pdhg) {
      spmv_t(n, &tc, vs, yb, g);
      ORC_PAR()
      for (int32_t j = 0; j < n; j++) zb[j] = cs[j] - g[j];
    }
    /* unscale the barred iterate and evaluate the KKT map on the original LP */
    ORC_PAR()
    for (int32_t j = 0; j < n; j++) {
      xo[j] = beta * Dc[j] * xb[j];
      double zz = gamma * zb[j] / Dc[j];
      if (zz > 0.0 && !isfinite(lp->xl[j])) zz = 0.0;
      if (zz < 0.0 && !isfinite(lp->xu[j])) zz = 0.0;
      zo[j] = zz;
    }
    ORC_PAR()
    for (int32_t i = 0; i < m; i++) yo[i] = gamma * Dr[i] * yb[i];
    kkt(lp, &tc, xo, yo, zo, last);
    have_out = 1;
    /* restart metric: fixed-point residual of the step, optionally in the
     * metric of the iteration (cross term with A(x_bar - x) = A x_t - A x_bar),
     * or the KKT error */
    double rho;
    if (pdhg || prm->restart_metric == 2) {
      rho = last[5];
    } else {
      double cross = 0.0;
      if (prm->restart_metric == 1) {
        spmv(m, lp->row_ptr, lp->col, vs, xb, pv);
        ORC_PAR(reduction(+ : cross))
        for (int32_t i = 0; i < m; i++) cross += (q[i] - pv[i]) * dyv[i];
      }
      rho = sqrt(fmax(0.0, dxx / sigma + lambda * sigma * dyy + 2.0 * cross));
    }

    int restart = 0;
    const int was_first = first_check;
    if (!isfinite(last[5])) {
      status = 3;  /* a residual is NaN or infinite: stop (no verdict) */
    } else if (last[5] <= prm->tol) {
      status = 0;
    } else if (prm->infeas_tol > 0.0 &&
               primal_infeasible(m, n, &tc, vs, los, his, xls, xus, dyv, prm->infeas_tol)) {
      status = 5;  /* the dual ray y_bar - y certifies primal infeasibility */
    } else if (prm->infeas_tol > 0.0 &&
               dual_infeasible(m, n, lp->row_ptr, lp->col, vs, cs, los, his, xls, xus, dxv, prm->infeas_tol)) {
      status = 6;  /* the direction x_bar - x certifies an unbounded primal */
    } else {
      /* restart rule (reading): sufficient / necessary / long */
      if (first_check) {
        rho0 = rho;
        first_check = 0;
        if ((double)k >= prm->restart_long * (double)t) restart = 1;
      } else {
        if (rho <= prm->restart_suff * rho0) restart = 1;
        else if (rho <= prm->restart_nec * rho0 && rho > rho_prev) restart = 1;
        else if ((double)k >= prm->restart_long * (double)t) restart = 1;
      }
      rho_prev = rho;
    }
    if (log && nlog < prm->log_cap) {
      orc_log* e = &log[nlog];
      e->iter = t;
      e->restart = restart;
      e->first = was_first;
      e->rp = last[0];
      e->rd = last[1];
      e->gap = last[2];
      e->pobj = last[3];
      e->dobj = last[4];
      e->rho = rho;
      e->sigma = sigma;
      e->rmap = last[6];
    }
    nlog++;
    /* an infeasibility verdict returns its certificate, unscaled like y or x */
    if (status == 5)
      for (int32_t i = 0; i < m; i++) yo[i] = gamma * Dr[i] * dyv[i];
    if (status == 6)
      for (int32_t j = 0; j < n; j++) xo[j] = beta * Dc[j] * dxv[j];
    if (status == 0 || status == 3 || status == 5 || status == 6) break;
    if (restart) {
      /* PDHG restarts from the average */
      if (pdhg) {
        memcpy(x, xb, sizeof(double) * (size_t)n);
        memcpy(y, yb, sizeof(double) * (size_t)m);
      }
      /* primal-weight update from the displacement since the last restart */
      double ddx = 0.0, ddy = 0.0;
      ORC_PAR(reduction(+ : ddx))
      for (int32_t j = 0; j < n; j++) ddx += (x[j] - x0[j]) * (x[j] - x0[j]);
      ORC_PAR(reduction(+ : ddy))
      for (int32_t i = 0; i < m; i++) ddy += (y[i] - y0[i]) * (y[i] - y0[i]);
      ddx = sqrt(ddx);
      ddy = sqrt(ddy);
      if (prm->sigma_update && ddx > 1e-10 && ddy > 1e-10) {
        double sig_new = ddx / (sqrt(lambda) * ddy);
        sigma = sqrt(sig_new * sigma); /* equal-weight geometric smoothing */
      }
      memcpy(x0, x, sizeof(double) * (size_t)n);
      memcpy(y0, y, sizeof(double) * (size_t)m);
      k = 0;
      if (prm->restart_ref == 1) rho0 = rho; /* decrease is measured from here */
      else first_check = 1;
      restarts++;
    }
  }

  if (have_out) {
    memcpy(x_out, xo, sizeof(double) * (size_t)n);
    memcpy(y_out, yo, sizeof(double) * (size_t)m);
    memcpy(z_out, zo, sizeof(double) * (size_t)n);
  }
  if (info) {
    info->iters = t;
    info->status = status;
    info->restarts = restarts;
    info->nlog = nlog;
    info->power_iters = piters;
    info->rp = last[0];
    info->rd = last[1];
    info->gap = last[2];
    info->pobj = last[3];
    info->dobj = last[4];
    info->kkt = last[5];
    info->lambda = lambda;
    info->sigma = sigma;
    info->beta = beta;
    info->gamma = gamma;
  }
  free(Dr); free(Dc); free(vs); free(cs); free(xls); free(xus); free(los); free(his);
  free(x); free(x0); free(xt); free(xb); free(zb); free(g); free(y); free(y0); free(yb);
  free(q); free(xo); free(yo); free(zo); free(dyv); free(pv);
  free(xbr); free(xavg); free(yavg); free(dxv);
  cols_free(&tc);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Sec. 4.1: Round and Algorithm 1                                         */
/* ---------------------------------------------------------------------- */
int32_t orc_round(double s, double tau) {
  if (s >= 1.0 - tau) return 1;
  if (s >= 0.0 && s <= tau) return 0;
  return -1;
}

int64_t orc_fix(int32_t G, int32_t T, const double* u, const double* v, const double* w,
                const int8_t* u_init, double tau, int32_t t_first, int8_t* fix_out) {
  int64_t nfixed = 0;
  int32_t* ru = (int32_t*)malloc(sizeof(int32_t) * (size_t)(T + 1));
  int32_t* rv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(T + 1));
  int32_t* rw = (int32_t*)malloc(sizeof(int32_t) * (size_t)(T + 1));
  for (int64_t e = 0; e < 3LL * G * T; e++) fix_out[e] = -1;
  for (int32_t g = 0; g < G; g++) {
    for (int32_t t = 0; t < T; t++) {
      ru[t] = orc_round(u[(int64_t)g * T + t], tau);
      rv[t] = orc_round(v[(int64_t)g * T + t], tau);
      rw[t] = orc_round(w[(int64_t)g * T + t], tau);
    }
    for (int32_t t = t_first; t < T; t++) {
      int32_t uprev = t > 0 ? ru[t - 1] : (int32_t)u_init[g];
      if (ru[t] == -1 || uprev == -1 || rv[t] == -1 || rw[t] == -1) break;
      if (ru[t] - uprev == rv[t] - rw[t] && rv[t] + rw[t] <= 1) {
        int64_t e = 3 * ((int64_t)g * T + t);
        fix_out[e + 0] = (int8_t)ru[t];
        fix_out[e + 1] = (int8_t)rv[t];
        fix_out[e + 2] = (int8_t)rw[t];
        nfixed++;
      } else {
        break;
      }
    }
  }
  free(ru);
  free(rv);
  free(rw);
  return nfixed;
}

/* ---------------------------------------------------------------------- */
/* Bound propagation (stands in for MILP-/LP-Presolve of Algorithm 2)      */
/* ---------------------------------------------------------------------- */
/* Activity range of one row over the bounds: the minimum and maximum of
 * sum_k a_k x_k for x within [xl, xu], with the finite parts summed in entry
 * order and the infinite contributions counted apart.                     */
static void row_activity(int64_t k0, int64_t k1, const int32_t* col, const double* val,
                         const double* xl, const double* xu, double* mn, double* mx,
                         int32_t* cmn, int32_t* cmx) {
  double s_mn = 0.0, s_mx = 0.0;
  int32_t c_mn = 0, c_mx = 0;
  for (int64_t k = k0; k < k1; k++) {
    double a = val[k];
    double lmin = a > 0.0 ? xl[col[k]] : xu[col[k]];
    double lmax = a > 0.0 ? xu[col[k]] : xl[col[k]];
    if (isinf(lmin)) c_mn++;
    else s_mn += a * lmin;
    if (isinf(lmax)) c_mx++;
    else s_mx += a * lmax;
  }
  *mn = s_mn;
  *mx = s_mx;
  *cmn = c_mn;
  *cmx = c_mx;
}

int32_t orc_propagate(int32_t m, int32_t n, const int64_t* rp, const int32_t* col,
                      const double* val, const double* lo, const double* hi, double* xl,
                      double* xu, const uint8_t* is_int, int32_t max_passes) {
  double* nlo = dalloc(n);
  double* nhi = dalloc(n);
  int32_t pass;
  int32_t result = 0;
  for (pass = 0; pass < max_passes; pass++) {
    memcpy(nlo, xl, sizeof(double) * (size_t)n);
    memcpy(nhi, xu, sizeof(double) * (size_t)n);
    /* Jacobi: every row uses the bounds of the previous pass */
    for (int32_t i = 0; i < m; i++) {
      double mn, mx;
      int32_t cmn, cmx;
      row_activity(rp[i], rp[i + 1], col, val, xl, xu, &mn, &mx, &cmn, &cmx);
      for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
        const int32_t j = col[k];
        const double a = val[k];
        const double lmin = a > 0.0 ? xl[j] : xu[j];
        const double lmax = a > 0.0 ? xu[j] : xl[j];
        /* from the row's upper bound: a x_j <= hi - (min activity of the rest);
         * a row whose maximum activity cannot exceed hi implies nothing */
        if (isfinite(hi[i]) && !(cmx == 0 && mx <= hi[i])) {
          int ok = isinf(lmin) ? (cmn == 1) : (cmn == 0);
          if (ok) {
            double rest = isinf(lmin) ? mn : mn - a * lmin;
            double b = (hi[i] - rest) / a;
            if (a > 0.0) { if (b < nhi[j]) nhi[j] = b; }
            else { if (b > nlo[j]) nlo[j] = b; }
          }
        }
        /* from the row's lower bound: a x_j >= lo - (max activity of the rest);
         * a row whose minimum activity cannot fall below lo implies nothing */
        if (isfinite(lo[i]) && !(cmn == 0 && mn >= lo[i])) {
          int ok = isinf(lmax) ? (cmx == 1) : (cmx == 0);
          if (ok) {
            double rest = isinf(lmax) ? mx : mx - a * lmax;
            double b = (lo[i] - rest) / a;
            if (a > 0.0) { if (b > nlo[j]) nlo[j] = b; }
            else { if (b < nhi[j]) nhi[j] = b; }
          }
        }
      }
    }
    int changed = 0;
    for (int32_t j = 0; j < n; j++) {
      double l = nlo[j], u = nhi[j];
      if (is_int[j]) {
        if (isfinite(u)) u = floor(u + 1e-6);
        if (isfinite(l)) l = ceil(l - 1e-6);
        if (l > xl[j]) { xl[j] = l; changed = 1; }
        if (u < xu[j]) { xu[j] = u; changed = 1; }
      } else {
        double tl = 1e-9 * fmax(1.0, isfinite(xl[j]) ? fabs(xl[j]) : 1.0);
        double tu = 1e-9 * fmax(1.0, isfinite(xu[j]) ? fabs(xu[j]) : 1.0);
        if (l > xl[j] + tl) { xl[j] = l; changed = 1; }
        if (u < xu[j] - tu) { xu[j] = u; changed = 1; }
      }
      if (xl[j] > xu[j] + 1e-6) result = -1 - pass;
    }
    if (result < 0) break;
    if (!changed) break;
  }
  free(nlo);
  free(nhi);
  if (result < 0) return result;
  return pass < max_passes ? pass + 1 : max_passes;
}

int orc_reduce(int32_t m, int32_t n, const int64_t* rp, const int32_t* col, const double* val,
               const double* c, const double* lo, const double* hi, const double* xl,
               const double* xu, int64_t* dims, int64_t* rp_r, int32_t* col_r, double* val_r,
               double* c_r, double* lo_r, double* hi_r, double* xl_r, double* xu_r,
               int32_t* row_map, int32_t* col_map, double* obj_const) {
  int32_t* newcol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t nr = 0;
  double oc = 0.0;
  for (int32_t j = 0; j < n; j++) {
    if (xl[j] == xu[j]) {
      newcol[j] = -1;
      oc += c[j] * xl[j];
    } else {
      newcol[j] = nr;
      col_map[nr] = j;
      c_r[nr] = c[j];
      xl_r[nr] = xl[j];
      xu_r[nr] = xu[j];
      nr++;
    }
  }
  int32_t mr = 0;
  int64_t kk = 0;
  int bad = 0;
  rp_r[0] = 0;
  for (int32_t i = 0; i < m; i++) {
    /* fold the fixed columns into the row bounds */
    double shift = 0.0;
    int64_t kept = 0;
    for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
      if (newcol[col[k]] < 0) shift += val[k] * xl[col[k]];
      else kept++;
    }
    double l = lo[i] - shift, u = hi[i] - shift;
    if (kept == 0) {
      if (l > 1e-6 * fmax(1.0, fabs(l)) || u < -1e-6 * fmax(1.0, fabs(u))) bad = 1;
      continue;
    }
    /* activity range over the free columns, in entry order */
    double mn = 0.0, mx = 0.0;
    int32_t cmn = 0, cmx = 0;
    for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
      const int32_t j = col[k];
      if (newcol[j] < 0) continue;
      const double a = val[k];
      const double lmin = a > 0.0 ? xl[j] : xu[j];
      const double lmax = a > 0.0 ? xu[j] : xl[j];
      if (isinf(lmin)) cmn++;
      else mn += a * lmin;
      if (isinf(lmax)) cmx++;
      else mx += a * lmax;
    }
    int lo_red = !isfinite(l) || (cmn == 0 && mn >= l);
    int hi_red = !isfinite(u) || (cmx == 0 && mx <= u);
    if (lo_red && hi_red) continue;
    row_map[mr] = i;
    lo_r[mr] = l;
    hi_r[mr] = u;
    for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
      int32_t nc = newcol[col[k]];
      if (nc < 0) continue;
      col_r[kk] = nc;
      val_r[kk] = val[k];
      kk++;
    }
    mr++;
    rp_r[mr] = kk;
  }
  dims[0] = mr;
  dims[1] = nr;
  dims[2] = kk;
  *obj_const = oc;
  free(newcol);
  return bad;
}
