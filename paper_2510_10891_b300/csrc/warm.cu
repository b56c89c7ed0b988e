// Warm start of the LP iteration from network predictions (scuc_ws_assemble,
// scuc_ws_targets) and the warm solve with cold start as its fallback
// (scuc_lp_solve_warm); declarations in include/scuc_ws.h.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/scuc_ws.h"
#include "lp.h"
#include "spmv.cuh"

namespace scuc {
namespace {

int grid_n(int64_t n) {
  const int64_t g = (n + kBlock - 1) / kBlock;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 148 * 16));
}

__device__ __forceinline__ double clamp_box(double v, double l, double u) { return v < l ? l : (v > u ? u : v); }

// a prediction as a value in [0, 1]; NaN counts as 0
__device__ __forceinline__ double unit_interval(float q) {
  const double v = (double)q;
  return v > 0.0 ? (v < 1.0 ? v : 1.0) : 0.0;
}

// x0 = projection of 0 onto [xl, xu]; y0 = 0
__global__ void k_ws_base(int n, int m, const double* __restrict__ xl, const double* __restrict__ xu,
                          double* __restrict__ x0, double* __restrict__ y0) {
  const int step = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += step) x0[j] = clamp_box(0.0, xl[j], xu[j]);
  if (y0)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += step) y0[i] = 0.0;
}

// unit-hour k = g*T + t: u, p' and (fill bits) v, w and the cost segments
__global__ void k_ws_units(scuc_ws_layout L, const float* __restrict__ pred, const double* __restrict__ xl,
                           const double* __restrict__ xu, double* __restrict__ x0) {
  const int GT = L.G * L.T;
  const int step = gridDim.x * blockDim.x;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < GT; k += step) {
    const int g = k / L.T, t = k - g * L.T;
    const double u = unit_interval(pred[3 * (int64_t)k]);
    const double r = fmin(unit_interval(pred[3 * (int64_t)k + 1]), u);
    const double p = __dmul_rn(r, L.p_cap[k]);
    int j = L.u_col[k];
    x0[j] = clamp_box(u, xl[j], xu[j]);
    j = L.p_col[k];
    x0[j] = clamp_box(p, xl[j], xu[j]);
    if (L.fill & SCUC_WS_FILL_VW) {
      const double prev = t > 0 ? unit_interval(pred[3 * (int64_t)(k - 1)]) : L.u_init[g];
      const double d = __dsub_rn(u, prev);
      j = L.v_col[k];
      x0[j] = clamp_box(d > 0.0 ? d : 0.0, xl[j], xu[j]);
      j = L.w_col[k];
      x0[j] = clamp_box(d < 0.0 ? -d : 0.0, xl[j], xu[j]);
    }
    if (L.fill & SCUC_WS_FILL_SEGMENTS) {
      double rem = p;
      for (int h = 0; h < L.nseg; h++) {
        const int64_t q = (int64_t)k * L.nseg + h;
        const double cap = __dmul_rn(L.seg_cap[q], u);
        const double sg = fmin(rem, cap);
        rem = __dsub_rn(rem, sg);
        j = L.seg_col[q];
        x0[j] = clamp_box(sg, xl[j], xu[j]);
      }
    }
  }
}

// price row q: y0 = price_scale * (mean of its members' predicted prices,
// summed in member order)
__global__ void k_ws_prices(scuc_ws_layout L, const float* __restrict__ pred, double* __restrict__ y0) {
  const int step = gridDim.x * blockDim.x;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < L.nprice; q += step) {
    const int a = L.price_ptr[q], b = L.price_ptr[q + 1];
    double s = 0.0;
    for (int e = a; e < b; e++) s = __dadd_rn(s, (double)pred[3 * (int64_t)L.price_member[e] + 2]);
    const double mean = b > a ? __ddiv_rn(s, (double)(b - a)) : 0.0;
    y0[L.price_row[q]] = __dmul_rn(L.price_scale, mean);
  }
}

// Y[k] = (x[u_col], x[p_col] / p_cap, y[unit_price_row] / price_scale)
__global__ void k_ws_targets(scuc_ws_layout L, const double* __restrict__ x, const double* __restrict__ y,
                             float* __restrict__ Y) {
  const int GT = L.G * L.T;
  const int step = gridDim.x * blockDim.x;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < GT; k += step) {
    const int row = L.unit_price_row ? L.unit_price_row[k] : -1;
    Y[3 * (int64_t)k] = (float)x[L.u_col[k]];
    Y[3 * (int64_t)k + 1] = (float)__ddiv_rn(x[L.p_col[k]], L.p_cap[k]);
    Y[3 * (int64_t)k + 2] = row >= 0 ? (float)__ddiv_rn(y[row], L.price_scale) : 0.f;
  }
}

// flag = 1 if some a[e] lies outside [lo, hi)
__global__ void k_check_range(const int32_t* __restrict__ a, int64_t cnt, int64_t lo, int64_t hi, int* flag) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += step)
    if (a[e] < lo || a[e] >= hi) atomicOr(flag, 1);
}

// flag = 1 unless 0 <= p[0] <= p[1] <= ... <= p[cnt-1]
__global__ void k_check_monotone(const int32_t* __restrict__ p, int64_t cnt, int* flag) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += step)
    if ((e == 0 && p[0] < 0) || (e > 0 && p[e] < p[e - 1])) atomicOr(flag, 1);
}

// Every index array a layout names is checked on the device before any
// kernel writes through it: an index out of range is an argument error.
int check_layout_indices(Handle& h, const scuc_ws_layout& L, bool assemble) {
  const int64_t GT = (int64_t)L.G * L.T;
  cudaStream_t s = h.work;
  if (!h.pt_flag) SCUC_TRY(h.alloc(&h.pt_flag, 2));
  SCUC_CUDA(cudaMemsetAsync(h.pt_flag, 0, 2 * sizeof(int), s));
  auto range = [&](const int32_t* a, int64_t cnt, int64_t lo, int64_t hi) {
    if (a && cnt > 0) k_check_range<<<grid_n(cnt), kBlock, 0, s>>>(a, cnt, lo, hi, h.pt_flag);
  };
  range(L.u_col, GT, 0, h.n);
  range(L.p_col, GT, 0, h.n);
  if (assemble) {
    if (L.fill & SCUC_WS_FILL_VW) {
      range(L.v_col, GT, 0, h.n);
      range(L.w_col, GT, 0, h.n);
    }
    if (L.fill & SCUC_WS_FILL_SEGMENTS) range(L.seg_col, GT * L.nseg, 0, h.n);
    if ((L.fill & SCUC_WS_FILL_PRICES) && L.nprice > 0) {
      range(L.price_row, L.nprice, 0, h.m);
      k_check_monotone<<<grid_n(L.nprice + 1), kBlock, 0, s>>>(L.price_ptr, L.nprice + 1, h.pt_flag);
    }
  } else {
    range(L.unit_price_row, GT, -1, h.m);
  }
  SCUC_CUDA(cudaGetLastError());
  int flag[2] = {0, 0};
  SCUC_CUDA(cudaMemcpyAsync(flag, h.pt_flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  SCUC_CUDA(cudaStreamSynchronize(s));
  if (flag[0]) {
    set_error("scuc_ws layout: an index array holds a column or row index out of range");
    return SCUC_E_INVALID;
  }
  if (assemble && (L.fill & SCUC_WS_FILL_PRICES) && L.nprice > 0) {
    int32_t nmem = 0;
    SCUC_CUDA(cudaMemcpyAsync(&nmem, L.price_ptr + L.nprice, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaStreamSynchronize(s));
    range(L.price_member, nmem, 0, GT);
    SCUC_CUDA(cudaGetLastError());
    SCUC_CUDA(cudaMemcpyAsync(flag, h.pt_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaStreamSynchronize(s));
    if (flag[0]) {
      set_error("scuc_ws layout: price_member holds a unit-hour out of range");
      return SCUC_E_INVALID;
    }
  }
  return SCUC_OK;
}

int check_layout(const Handle& h, const scuc_ws_layout* L, bool assemble) {
  if (!L || L->G < 0 || L->T < 0 || (int64_t)L->G * L->T > (int64_t)h.n) {
    set_error("scuc_ws layout: invalid G, T");
    return SCUC_E_INVALID;
  }
  if (L->G * L->T == 0) return SCUC_OK;
  if (!L->u_col || !L->p_col || !L->p_cap) {
    set_error("scuc_ws layout: u_col, p_col and p_cap are required");
    return SCUC_E_INVALID;
  }
  if (assemble) {
    if ((L->fill & SCUC_WS_FILL_VW) && (!L->v_col || !L->w_col || !L->u_init)) {
      set_error("scuc_ws layout: FILL_VW needs v_col, w_col and u_init");
      return SCUC_E_INVALID;
    }
    if ((L->fill & SCUC_WS_FILL_SEGMENTS) && (L->nseg < 0 || L->nseg > 8 || (L->nseg > 0 && (!L->seg_col || !L->seg_cap)))) {
      set_error("scuc_ws layout: FILL_SEGMENTS needs 0 <= nseg <= 8, seg_col and seg_cap");
      return SCUC_E_INVALID;
    }
    if ((L->fill & SCUC_WS_FILL_PRICES) &&
        (L->nprice < 0 || (L->nprice > 0 && (!L->price_row || !L->price_ptr || !L->price_member)))) {
      set_error("scuc_ws layout: FILL_PRICES needs price_row, price_ptr and price_member");
      return SCUC_E_INVALID;
    }
  } else if (L->unit_price_row && !(L->price_scale != 0.0 && std::isfinite(L->price_scale))) {
    set_error("scuc_ws layout: price_scale must be finite and non-zero");
    return SCUC_E_INVALID;
  }
  return SCUC_OK;
}

}  // namespace

}  // namespace scuc

using scuc::Handle;

extern "C" {

int scuc_ws_assemble(scuc_lp* lp, const scuc_ws_layout* L, const float* pred_dev, double* x0_dev, double* y0_dev) {
  if (!lp || !lp->h || !x0_dev || (!pred_dev && L && L->G * L->T > 0)) {
    scuc::set_error("scuc_ws_assemble: null argument");
    return SCUC_E_INVALID;
  }
  Handle& h = *lp->h;
  SCUC_TRY(scuc::check_layout(h, L, true));
  SCUC_TRY(h.enter());
  SCUC_TRY(scuc::check_layout_indices(h, *L, true));
  cudaStream_t s = h.work;
  scuc::k_ws_base<<<scuc::grid_n(std::max(h.m, h.n)), scuc::kBlock, 0, s>>>(h.n, h.m, h.xl, h.xu, x0_dev, y0_dev);
  const int GT = L->G * L->T;
  if (GT > 0) scuc::k_ws_units<<<scuc::grid_n(GT), scuc::kBlock, 0, s>>>(*L, pred_dev, h.xl, h.xu, x0_dev);
  if (y0_dev && (L->fill & SCUC_WS_FILL_PRICES) && L->nprice > 0)
    scuc::k_ws_prices<<<scuc::grid_n(L->nprice), scuc::kBlock, 0, s>>>(*L, pred_dev, y0_dev);
  SCUC_CUDA(cudaGetLastError());
  SCUC_CUDA(cudaStreamSynchronize(s));
  return h.leave();
}

int scuc_ws_targets(scuc_lp* lp, const scuc_ws_layout* L, const double* x_dev, const double* y_dev, float* Y_dev) {
  if (!lp || !lp->h || !L || !x_dev || !Y_dev || (L->unit_price_row && !y_dev)) {
    scuc::set_error("scuc_ws_targets: null argument");
    return SCUC_E_INVALID;
  }
  Handle& h = *lp->h;
  SCUC_TRY(scuc::check_layout(h, L, false));
  const int GT = L->G * L->T;
  if (GT == 0) return SCUC_OK;
  SCUC_TRY(h.enter());
  SCUC_TRY(scuc::check_layout_indices(h, *L, false));
  cudaStream_t s = h.work;
  scuc::k_ws_targets<<<scuc::grid_n(GT), scuc::kBlock, 0, s>>>(*L, x_dev, y_dev, Y_dev);
  SCUC_CUDA(cudaGetLastError());
  SCUC_CUDA(cudaStreamSynchronize(s));
  return h.leave();
}

void scuc_default_warm_params(scuc_warm_params* w) {
  if (!w) return;
  w->warm_max_iter = 0;
  w->first_check = 1;
  w->cold_first_kkt = 0.0;
}

int scuc_lp_solve_warm(scuc_lp* lp, const scuc_solve_params* p, const double* x0, const double* y0,
                       const scuc_warm_params* wp_in, double* x_out, double* y_out, double* z_out,
                       scuc_solve_info* info) {
  if (!lp || !lp->h || !p || !x0) {
    scuc::set_error("scuc_lp_solve_warm: null argument");
    return SCUC_E_INVALID;
  }
  scuc_warm_params wp;
  scuc_default_warm_params(&wp);
  if (wp_in) wp = *wp_in;
  Handle& h = *lp->h;
  scuc_solve_params pw = *p;
  double ref = wp.cold_first_kkt;
  scuc_solve_info ir;
  memset(&ir, 0, sizeof(ir));
  if (wp.first_check && !(ref > 0.0)) {
    // the cold start's first check: one period from the cold point
    scuc_solve_params pr = *p;
    pr.max_iter = p->check_every;
    SCUC_TRY(h.solve(pr, nullptr, nullptr, x_out, y_out, z_out, &ir));
    if (ir.status == SCUC_ST_OPTIMAL) {
      if (info) {
        *info = ir;
        info->ref_iters = ir.iters;
        info->cold_first_kkt = ir.kkt;
      }
      return SCUC_OK;
    }
    ref = ir.kkt;
    // the power method is deterministic: reuse its lambda instead of repeating it
    if (!(pw.lambda_in > 0.0)) pw.lambda_in = ir.lambda;
  }
  if (wp.warm_max_iter > 0) pw.max_iter = std::min<int64_t>(p->max_iter, wp.warm_max_iter);
  scuc_solve_info iw;
  // the reference period left the scaled data of this same model in place
  SCUC_TRY(h.solve(pw, x0, y0, x_out, y_out, z_out, &iw, wp.first_check ? ref : 0.0, ir.iters > 0));
  auto add = [](scuc_solve_info& a, const scuc_solve_info& b) {
    a.iters += b.iters;
    a.iters_fp32 += b.iters_fp32;
    a.setup_ms += b.setup_ms;
    a.solve_ms += b.solve_ms;
    a.launches += b.launches;
    a.ms_dual_spmv += b.ms_dual_spmv;
    a.ms_primal_spmv += b.ms_primal_spmv;
    a.n_dual_spmv += b.n_dual_spmv;
    a.n_primal_spmv += b.n_primal_spmv;
    a.ms_dual_spmv_f32 += b.ms_dual_spmv_f32;
    a.ms_primal_spmv_f32 += b.ms_primal_spmv_f32;
    a.n_dual_spmv_f32 += b.n_dual_spmv_f32;
    a.n_primal_spmv_f32 += b.n_primal_spmv_f32;
  };
  if (iw.status == SCUC_ST_OPTIMAL) {
    if (info) {
      scuc_solve_info out = iw;
      add(out, ir);
      out.power_iters = iw.power_iters + ir.power_iters;
      out.warm_iters = 0;
      out.ref_iters = ir.iters;
      out.cold_first_kkt = ref;
      *info = out;
    }
    return SCUC_OK;
  }
  // rejected: cold solve with the same lambda
  scuc_solve_params pc = *p;
  if (!(pc.lambda_in > 0.0)) pc.lambda_in = iw.lambda;
  scuc_solve_info ic;
  SCUC_TRY(h.solve(pc, nullptr, nullptr, x_out, y_out, z_out, &ic, 0.0, true));
  if (info) {
    scuc_solve_info out = ic;
    if (ic.status == SCUC_ST_OPTIMAL) out.status = SCUC_ST_FALLBACK_COLD;
    add(out, iw);
    add(out, ir);
    out.power_iters = iw.power_iters + ir.power_iters;
    out.warm_iters = iw.iters;
    out.ref_iters = ir.iters;
    out.cold_first_kkt = ref;
    *info = out;
  }
  return SCUC_OK;
}

}  // extern "C"
