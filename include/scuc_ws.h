/* Learned warm start for the SCUC LP relaxation.
 *
 * The paper has no learned component: its first-order LP solves always start
 * from zero (Eq. 9 iterates from a given (x^0, y^0)).  This part predicts,
 * for every generator-hour (g, t), the relaxed commitment u_{g,t}, the output
 * above minimum p'_{g,t} as a fraction of P^U_g - P^L_g (Eq. 3), and the
 * price of the balance row of Eq. 6 that the unit feeds, and turns those
 * predictions into a starting point (x^0, y^0) of the iteration of Eq. 9.
 *
 * Network: a multilayer perceptron, dims[0] inputs -> ... -> 3 outputs, ReLU
 * between layers.  Weights and activations are BF16 on the tensor cores with
 * FP32 accumulation; master weights, biases and Adam moments are FP32.
 * Outputs: o_0 -> u = sigmoid(o_0); o_1 -> r = sigmoid(o_1) (p' fraction);
 * o_2 -> price (identity).
 *
 * Loss of one sample with targets (u*, r*, q*), averaged over a batch:
 *   softplus(o_0) - u* o_0                (cross-entropy of sigmoid(o_0))
 *   + w_dispatch (sigmoid(o_1) - r*)^2
 *   + w_price (o_2 - q*)^2
 *
 * Conventions as in scuc_lp.h: the return code is the error, messages from
 * scuc_last_error(), inputs are caller-owned and never retained.  Pointers
 * named *_dev are device pointers on the device that was current at
 * scuc_ws_create; every other pointer is host memory.  A scuc_ws handle is
 * not thread-safe.  All device work of a handle runs on the stream given at
 * creation, and each call returns after that work has completed unless it
 * says otherwise.                                                            */
#ifndef SCUC_WS_H
#define SCUC_WS_H

#include "scuc_lp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scuc_ws scuc_ws;

typedef struct {
  float lr;          /* Adam step size (1e-3)                                */
  float beta1;       /* 0.9                                                  */
  float beta2;       /* 0.999                                                */
  float eps;         /* 1e-8                                                 */
  float w_dispatch;  /* weight of the p' fraction term (1)                   */
  float w_price;     /* weight of the price term (1)                         */
} scuc_ws_train_params;

void scuc_ws_default_train_params(scuc_ws_train_params* p);

/* nlayers linear layers with widths dims[0..nlayers]; dims[nlayers] must be
 * 3 and every width 1..4096.  Parameters start at zero (load them with
 * scuc_ws_set_params), the input standardisation at mean 0, scale 1.
 * cuda_stream: the stream of all later work (NULL: the legacy stream).     */
int scuc_ws_create(scuc_ws** out, int32_t nlayers, const int32_t* dims, void* cuda_stream);

/* Number of parameters: sum over layers of dims[l]*dims[l+1] + dims[l+1].   */
int scuc_ws_num_params(const scuc_ws* ws, int64_t* count);

/* Parameter vector (host, FP32): for each layer l in order, W_l row-major
 * [dims[l] x dims[l+1]] (input index major), then b_l [dims[l+1]].  Setting
 * the parameters also clears the Adam moments and step count.               */
int scuc_ws_set_params(scuc_ws* ws, const float* params);
int scuc_ws_get_params(const scuc_ws* ws, float* params);

/* Input standardisation x_s = (x - mean) / scale, applied to raw features
 * before the first layer.  mean[dims[0]], scale[dims[0]] (host, scale > 0). */
int scuc_ws_set_input_norm(scuc_ws* ws, const float* mean, const float* scale);

/* Predictions for rows samples: X_dev[rows x dims[0]] raw features (FP32,
 * row-major) -> out_dev[rows x 3] = (u, r, price) after the output maps.     */
int scuc_ws_predict(scuc_ws* ws, const float* X_dev, int32_t rows, float* out_dev);

/* Mean loss over rows samples and its gradient with respect to every
 * parameter, with no update.  Y_dev[rows x 3] targets (u*, r*, q*).
 * grads: host FP32 in the parameter layout (NULL: not returned);
 * loss: host (NULL: not returned).  The gradients are those of the BF16
 * network: BF16 weights and activations, FP32 accumulation.                */
int scuc_ws_gradients(scuc_ws* ws, const float* X_dev, const float* Y_dev, int32_t rows,
                      const scuc_ws_train_params* p, float* grads, double* loss);

/* steps Adam steps of batch samples each.  Step s uses the samples
 * idx_dev[s*batch .. s*batch + batch - 1] (device int32, each < nsamples);
 * the caller draws them.  X_dev[nsamples x dims[0]], Y_dev[nsamples x 3].
 * losses: host double[steps] receiving each step's batch loss (before the
 * step's update), or NULL.  Deterministic: the same inputs give the same
 * parameters bit for bit.                                                  */
int scuc_ws_train(scuc_ws* ws, const float* X_dev, const float* Y_dev, int64_t nsamples,
                  const int32_t* idx_dev, int32_t batch, int32_t steps, const scuc_ws_train_params* p,
                  double* losses);

/* Kernels of the forward products (no counterpart in the paper; both are
 * BF16 operands with FP32 accumulation, summed in different orders):
 * SCUC_WS_GEMM_TCGEN05 (the default) runs the hidden layers whose input
 * width is a multiple of 64 up to 256 and whose output width is a multiple
 * of 16 up to 256 on tcgen05 (TMA loads, tensor-memory accumulator, bias and
 * activation in its epilogue) and the other layers on mma.sync;
 * SCUC_WS_GEMM_MMA_SYNC runs every layer on mma.sync.  A bounded wait of the
 * tcgen05 kernel that runs out makes predict / gradients / train return
 * SCUC_E_DEVICE_TIMEOUT.  SCUC_E_INVALID for another kind.               */
enum { SCUC_WS_GEMM_TCGEN05 = 0, SCUC_WS_GEMM_MMA_SYNC = 1 };
int scuc_ws_set_gemm(scuc_ws* ws, int32_t kind);

void scuc_ws_destroy(scuc_ws* ws);

/* ------------------------------------------------------------------------
 * From predictions to a starting point, and from solutions to targets.
 * ------------------------------------------------------------------------ */
enum {
  SCUC_WS_FILL_VW = 1,        /* v_t = max(u_t - u_{t-1}, 0), w_t = max(u_{t-1} - u_t, 0)
                                 (Eq. 1 with u_{g,0} = u_init[g]); else 0     */
  SCUC_WS_FILL_SEGMENTS = 2,  /* p' split over the cost segments in index order,
                                 segment h capped at seg_cap*u (Eq. 5); else 0 */
  SCUC_WS_FILL_PRICES = 4     /* duals of the price rows; else 0              */
};

/* All pointers are device pointers.  Unit-hour k = g*T + t.                 */
typedef struct {
  int32_t G, T;
  int32_t nseg;                 /* cost segments per unit-hour (0..8)        */
  int32_t fill;                 /* SCUC_WS_FILL_* bits                       */
  const int32_t* u_col;         /* [G*T] column of u_{g,t}                   */
  const int32_t* v_col;         /* [G*T] column of v_{g,t} (FILL_VW)         */
  const int32_t* w_col;         /* [G*T] column of w_{g,t} (FILL_VW)         */
  const int32_t* p_col;         /* [G*T] column of p'_{g,t}                  */
  const int32_t* seg_col;       /* [G*T*nseg] segment columns (FILL_SEGMENTS) */
  const double* p_cap;          /* [G*T] P^U - P^L in LP units (> 0)         */
  const double* seg_cap;        /* [G*T*nseg] segment widths in LP units     */
  const double* u_init;         /* [G] commitment before the first hour      */
  const int32_t* unit_price_row;/* [G*T] row whose dual is the price of unit-hour k,
                                   -1: none (targets)                         */
  int32_t nprice;               /* rows that receive a dual (FILL_PRICES)    */
  const int32_t* price_row;     /* [nprice] LP row                           */
  const int32_t* price_ptr;     /* [nprice + 1] ranges of price_member       */
  const int32_t* price_member;  /* unit-hours whose predicted prices average
                                   into each row, in summation order         */
  double price_scale;           /* dual of a price row = price_scale * price */
} scuc_ws_layout;

/* Starting point from predictions pred_dev[G*T x 3] (as scuc_ws_predict
 * writes them).  x0_dev[n]: every column starts at the projection of 0 onto
 * [xl, xu] (the handle's current bounds); then u = clamp(u_pred, 0, 1),
 * p' = min(r_pred, u) * p_cap, and the FILL_* parts; each written value is
 * projected onto [xl_j, xu_j].  y0_dev[m] (may be NULL): 0, and with
 * FILL_PRICES each price row gets price_scale times the mean of its members'
 * predicted prices.  Queued on the handle's stream; returns after it ends. */
int scuc_ws_assemble(scuc_lp* lp, const scuc_ws_layout* L, const float* pred_dev, double* x0_dev,
                     double* y0_dev);

/* Training targets from a solution (unscaled, device): Y_dev[G*T x 3] =
 * (x[u_col], x[p_col] / p_cap, y[unit_price_row] / price_scale), the price 0
 * where unit_price_row is -1.  Queued on the handle's stream; returns after
 * it ends.                                                                 */
int scuc_ws_targets(scuc_lp* lp, const scuc_ws_layout* L, const double* x_dev, const double* y_dev,
                    float* Y_dev);

/* Solve from a warm start with cold start as the fallback.
 *  x0, y0: the warm point (device pointers when p->device_ptrs, else host;
 *    y0 may be NULL).
 *  The warm run is rejected
 *   - (first_check) if the KKT measure at its first check, max(r_p, r_d,
 *     gap) after check_every iterations, is not below the cold start's at
 *     its first check.  That reference is cold_first_kkt when it is > 0,
 *     else it is measured by one check period from the cold start (those
 *     iterations are counted in info->iters and info->ref_iters, and the
 *     lambda of that run is reused);
 *   - or if it has not reached p->tol after warm_max_iter iterations
 *     (<= 0: p->max_iter).
 *  A rejected warm run is followed by a cold solve with *p; info->status is
 *  then SCUC_ST_FALLBACK_COLD when the cold solve reaches tol (its own status
 *  otherwise).  info->iters counts the iterations of every run, and
 *  info->warm_iters those of a rejected warm run.
 *  Outputs as in scuc_lp_solve.                                             */
typedef struct {
  int64_t warm_max_iter;  /* 0: p->max_iter                                 */
  int32_t first_check;    /* 1: apply the first-check test                  */
  double cold_first_kkt;  /* > 0: the cold start's first-check KKT measure,
                             known to the caller; 0: measure it             */
} scuc_warm_params;

void scuc_default_warm_params(scuc_warm_params* w);

int scuc_lp_solve_warm(scuc_lp* lp, const scuc_solve_params* p, const double* x0, const double* y0,
                       const scuc_warm_params* wp, double* x_out, double* y_out, double* z_out,
                       scuc_solve_info* info);

#ifdef __cplusplus
}
#endif
#endif
