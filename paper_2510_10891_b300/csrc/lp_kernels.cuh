// HPR iteration kernels (Eq. 9) with the dual/primal epilogues fused into the
// SpMVs, the KKT-check SpMVs, and the single-block decide kernel.
#pragma once
#include "spmv.cuh"

namespace scuc {

struct DevLP {
  int m, n;
  // A (rows) and A^T (columns) in CSR, 32-bit indices
  const int *rp, *col, *rpt, *colt;
  const double *vs, *vst;      // scaled values  A_hat = D_r A D_c
  const float *vs32, *vst32;   // FP32 copies (mixed precision)
  const double *val, *valt;    // unscaled values
  // scaled problem data
  const double *c, *xl, *xu, *lo, *hi, *Dr, *Dc;
  // iterates
  double *x, *x0, *xt, *xbar, *zbar, *y, *y0, *ybar;
  float *xt32, *y32;
  double *qchk, *dychk;        // A x_t and y_bar - y at a check iteration
  double* dxchk;               // x_bar - x at a check iteration (infeasibility detection)
  const double* coef;          // Halpern weights {1/(k+2), (k+1)/(k+2)} per period slot
  double* coef_w;              // same buffer, written by the decide kernel
  double* gsum;                // A^T y of the primal step in FP64 phases
  float* gsum32;               // ... in FP32 phases (LPs of a batch may be in different phases)
  // partial sums
  double *partP, *partD, *partRA, *partRT;
  int epi_gx;                  // blocks per LP of the primal epilogue (partP: epi_gx * nlp slots)
  Partition pA, pT;
  Sell sT;                     // sliced ELL copy of A^T (one LP; nslice = 0: none)
  Sell sA;                     // sliced ELL copy of A's rows of <= kSellMaxLen nonzeros (one LP)
  Ctrl* ctrl;
  scuc_check_log* log;
  // A batch of nlp LPs stored as one block-diagonal LP (nlp = 1: one LP).
  // Blocks of pA / pT never span two LPs: blkA / blkT give the LP of each
  // block (nullptr: LP 0), ablk0 / tblk0 the first block of each LP, row0 /
  // col0 its first row and column.  Per-LP state: ctrl[lp], coef + lp *
  // coef_stride, log + lp * log_stride.
  int nlp;
  const int *blkA, *blkT, *ablk0, *tblk0, *row0, *col0;
  int coef_stride, log_stride;
};

// range [a, b) of LP lp in an offsets array (nullptr: the whole range)
__device__ __forceinline__ void lp_range(const int* off, int lp, int total, int& a, int& b) {
  if (off) {
    a = off[lp];
    b = off[lp + 1];
  } else {
    a = 0;
    b = total;
  }
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ double clampd(double v, double l, double u) {
  return v < l ? l : (v > u ? u : v);
}

// The same order tests on the integer pipes: non-NaN doubles ordered as
// signed 64-bit keys (-0 sorts just below +0, which changes at most the sign
// of a zero result).  The iteration epilogues are bound by B300's FP64 pipe.
__device__ __forceinline__ long long dkey(double v) {
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : b ^ 0x7fffffffffffffffLL;
}
__device__ __forceinline__ double clamp_k(double v, double l, double u) {
  const long long k = dkey(v);
  return k < dkey(l) ? l : (k > dkey(u) ? u : v);
}
__device__ __forceinline__ double max0(double v) { return __double_as_longlong(v) > 0 ? v : 0.0; }
__device__ __forceinline__ double min0(double v) { return __double_as_longlong(v) < 0 ? v : 0.0; }

// Kernels and their helpers have internal linkage: every translation unit
// that launches them compiles its own copy.
namespace {

// Precision of the products in an iteration kernel: kPrecRuntime reads each
// LP's phase from its control block (batches, whose LPs switch at different
// times); kPrecF32 / kPrecF64 are compiled for one phase (one LP, whose phase
// picks the kernels: a graph conditional, or the host between periods), so
// each gets its own register allocation.
constexpr int kPrecRuntime = 0, kPrecF32 = 1, kPrecF64 = 2;

__device__ __forceinline__ bool phase64(const Ctrl* c, int prec) {
  return prec == kPrecRuntime ? c->fp64_phase != 0 : prec == kPrecF64;
}

// ---------------------------------------------------------------------------
// chunk launches of the long rows (one LP; batches have no long rows)
// ---------------------------------------------------------------------------
constexpr int kChunksPrimal = 0, kChunksDual = 1, kChunksResPrimal = 2, kChunksResDual = 3, kChunksInfRows = 4,
              kChunksInfCols = 5;

// Chunk sums for the next main launch: A^T y (primal step) or A x_t (dual
// step) in the phase's precision, A x_bar / A^T y_bar (checks) and the
// certificate products A (x_bar - x) / A^T (y_bar - y) in FP64.
template <int KIND, int PREC>
__global__ void __launch_bounds__(kBlock) k_chunks_iter(DevLP L) {
  const Ctrl* ctrl = L.ctrl;
  if (ctrl->done) return;
  const bool fp64 = phase64(ctrl, PREC);
  if (KIND == kChunksPrimal) {
    if (fp64) chunk_warp<double>(L.colt, L.vst, L.y, L.pT);
    else chunk_warp<float>(L.colt, L.vst32, L.y32, L.pT);
  } else if (KIND == kChunksDual) {
    if (fp64) chunk_warp<double>(L.col, L.vs, L.xt, L.pA);
    else chunk_warp<float>(L.col, L.vs32, L.xt32, L.pA);
  } else if (KIND == kChunksResPrimal) {
    chunk_warp<double>(L.col, L.vs, L.xbar, L.pA);
  } else if (KIND == kChunksResDual) {
    chunk_warp<double>(L.colt, L.vst, L.ybar, L.pT);
  } else if (KIND == kChunksInfRows) {
    chunk_warp<double>(L.col, L.vs, L.dxchk, L.pA);
  } else {
    chunk_warp<double>(L.colt, L.vst, L.dychk, L.pT);
  }
}

// ---------------------------------------------------------------------------
// primal step over A^T y: x_bar = Pi_K(x + sigma (g - c)), reflection, Halpern
// ---------------------------------------------------------------------------
template <bool CHECK>
struct PrimalEpi {
  const DevLP& L;
  double sigma, wa, wb;
  bool fp64;
  bool pdhg;  // restarted PDHG with ergodic averaging: x^{k+1} = x_bar, running average in xbar
  bool ray;   // infeasibility detection: store x_bar - x on checks
  double acc[4];
  double xj, cj, xlj, xuj, x0j;  // the column's operands, loaded before its sum
  __device__ void load(int j) {
    xj = L.x[j];
    cj = L.c[j];
    xlj = L.xl[j];
    xuj = L.xu[j];
    x0j = L.x0[j];
  }
  __device__ void row(int j, double g) {
    const double v = xj + sigma * (g - cj);
    const double xb = clamp_k(v, xlj, xuj);
    const double xt = 2.0 * xb - xj;
    double xn, xa = 0.0;
    if (pdhg) {  // weights {1/(k+1), k/(k+1)} of the running average (rounded as written); k = 0 starts it
      xn = xb;
      xa = wb == 0.0 ? xb : __dadd_rn(__dmul_rn(wa, xb), __dmul_rn(wb, L.xbar[j]));
      L.xbar[j] = xa;
    } else {
      xn = wa * x0j + wb * xt;
    }
    L.x[j] = xn;
    if (fp64) L.xt[j] = xt;
    else L.xt32[j] = (float)xt;
    if (CHECK) {
      if (ray) L.dxchk[j] = xb - xj;
      acc[0] += (xb - xj) * (xb - xj);
      if (pdhg) {  // the checked point is the average; its z comes with A^T y_avg
        acc[1] += (xa - x0j) * (xa - x0j);
        acc[2] += cj * xa;
        return;
      }
      double zb = (xb - v) / sigma;
      if (zb > 0.0 && !isfinite(xlj)) zb = 0.0;
      if (zb < 0.0 && !isfinite(xuj)) zb = 0.0;
      L.xbar[j] = xb;
      L.zbar[j] = zb;
      acc[1] += (xn - x0j) * (xn - x0j);
      acc[2] += cj * xb;
      if (zb > 0.0) acc[3] += xlj * zb;
      else if (zb < 0.0) acc[3] += xuj * zb;
    }
  }
};

// g = A^T y (the primal step's product), stored for the elementwise epilogue
template <typename VT>
struct GStoreEpi {
  VT* g;
  __device__ void load(int) {}
  __device__ void row(int r, VT a) { g[r] = a; }
};

template <int PREC>
__global__ void __launch_bounds__(kBlock) k_primal_sum(DevLP L) {
  extern __shared__ __align__(128) unsigned char smem[];
  const BlockPlan bp = spmv_plan<false>(L.pT);  // issued together with the control loads
  const Ctrl* ctrl = L.ctrl + (L.blkT ? L.blkT[blockIdx.x] : 0);
  if (ctrl->done) return;
  if (phase64(ctrl, PREC)) {
    GStoreEpi<double> e{L.gsum};
    spmv_run<double, GStoreEpi<double>, true>(bp, L.rpt, L.colt, L.vst, L.y, L.pT, smem, e);
  } else {
    GStoreEpi<float> e{L.gsum32};
    spmv_run<float, GStoreEpi<float>, true>(bp, L.rpt, L.colt, L.vst32, L.y32, L.pT, smem, e);
  }
}

// Sum of lane `lane`'s row of slice sl of a sliced ELL copy (Sell), in the
// row's entry order.  FP32 values: batches of 16 entries per lane (one
// 8-byte {column, value} load each, all issued before the products), even
// and odd entries in two accumulators, the last partial batch predicated;
// FP64 values: batches of 8 into one accumulator (the FP64 pipe, not the
// loads, bounds the FP64 products).
__device__ __forceinline__ float sell_sum(const Sell& S, const float* __restrict__ x, int sl, int lane) {
  constexpr int U = 16;
  const int steps = S.sptr[sl + 1] - S.sptr[sl];
  const int2* __restrict__ cv = S.cv32 + (int64_t)S.sptr[sl] * 32 + lane;
  float a0 = 0.f, a1 = 0.f;
  int k = 0;
  for (; k + U <= steps; k += U) {
    int2 e[U];
#pragma unroll
    for (int u = 0; u < U; u++) e[u] = ldcs(cv + (int64_t)(k + u) * 32);
#pragma unroll
    for (int u = 0; u < U; u += 2) {
      a0 = fma_t(__int_as_float(e[u].y), ldg(x + e[u].x), a0);
      a1 = fma_t(__int_as_float(e[u + 1].y), ldg(x + e[u + 1].x), a1);
    }
  }
  if (k < steps) {
    int2 e[U];
#pragma unroll
    for (int u = 0; u < U; u++) e[u] = k + u < steps ? ldcs(cv + (int64_t)(k + u) * 32) : make_int2(-1, 0);
#pragma unroll
    for (int u = 0; u < U; u += 2) {
      if (e[u].x >= 0) a0 = fma_t(__int_as_float(e[u].y), ldg(x + e[u].x), a0);
      if (e[u + 1].x >= 0) a1 = fma_t(__int_as_float(e[u + 1].y), ldg(x + e[u + 1].x), a1);
    }
  }
  return a0 + a1;
}

// The same sum on the compressed form (Sell::compressed): batches of 8 step
// pairs (16 entries) per lane, one 8-byte value pair and one 4-byte offset
// pair per load, step k's column = (k < kjump ? base0 : base1) + offset;
// even steps into one accumulator, odd steps into the other, as above (the
// same sum; a padded step of an odd-length slice adds a zero product).
__device__ __forceinline__ float sell_sum_c(const Sell& S, const float* __restrict__ x, int sl, int lane,
                                            int4 rec) {
  constexpr int U = 8;
  const int np = S.pptr[sl + 1] - S.pptr[sl];
  const int64_t base = (int64_t)S.pptr[sl] * 32 + lane;
  const float2* __restrict__ vp = S.v2 + base;
  const unsigned* __restrict__ op = S.o2 + base;
  const int b0 = rec.y, b1 = rec.z, kj = rec.w;
  float a0 = 0.f, a1 = 0.f;
  int p = 0;
  for (; p + U <= np; p += U) {
    float2 v[U];
    unsigned o[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      v[u] = ldcs(vp + (int64_t)(p + u) * 32);
      o[u] = ldcs(op + (int64_t)(p + u) * 32);
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int k = 2 * (p + u);
      const int c0 = (k < kj ? b0 : b1) + (int)(o[u] & 0xffffu);
      const int c1 = (k + 1 < kj ? b0 : b1) + (int)(o[u] >> 16);
      a0 = fma_t(v[u].x, ldg(x + c0), a0);
      a1 = fma_t(v[u].y, ldg(x + c1), a1);
    }
  }
  if (p < np) {
    float2 v[U];
    unsigned o[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      v[u] = p + u < np ? ldcs(vp + (int64_t)(p + u) * 32) : make_float2(0.f, 0.f);
      o[u] = p + u < np ? ldcs(op + (int64_t)(p + u) * 32) : 0u;
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (p + u < np) {
        const int k = 2 * (p + u);
        const int c0 = (k < kj ? b0 : b1) + (int)(o[u] & 0xffffu);
        const int c1 = (k + 1 < kj ? b0 : b1) + (int)(o[u] >> 16);
        a0 = fma_t(v[u].x, ldg(x + c0), a0);
        a1 = fma_t(v[u].y, ldg(x + c1), a1);
      }
    }
  }
  return a0 + a1;
}

// FP32 sum of lane `lane`'s row of slice sl from the FP32 form the copy
// holds; r receives the row (-1: none).
__device__ __forceinline__ float sell_sum32(const Sell& S, const float* __restrict__ x, int sl, int lane, int& r) {
  if (S.compressed) {
    const int4 rec = S.lrec[(size_t)sl * 32 + lane];
    r = rec.x;
    return sell_sum_c(S, x, sl, lane, rec);
  }
  r = S.rows[(size_t)sl * 32 + lane];
  return sell_sum(S, x, sl, lane);
}

__device__ __forceinline__ double sell_sum(const Sell& S, const double* __restrict__ x, int sl, int lane) {
  constexpr int U = 8;
  const int steps = S.sptr[sl + 1] - S.sptr[sl];
  const int64_t base = (int64_t)S.sptr[sl] * 32 + lane;
  const int* __restrict__ cc = S.col + base;
  const double* __restrict__ vv = S.v64 + base;
  double a = 0.0;
  int k = 0;
  for (; k + U <= steps; k += U) {
    int c[U];
    double v[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      c[u] = ldcs(cc + (int64_t)(k + u) * 32);
      v[u] = ldcs(vv + (int64_t)(k + u) * 32);
    }
#pragma unroll
    for (int u = 0; u < U; u++) a = fma_t(v[u], ldg(x + c[u]), a);
  }
  for (; k < steps; k++) a = fma_t(ldcs(vv + (int64_t)k * 32), ldg(x + ldcs(cc + (int64_t)k * 32)), a);
  return a;
}

// g = A^T y on the sliced ELL copy of A^T (one LP): blocks [0, nsb) take one
// slice of 32 columns per warp, one column per lane; the blocks after them
// give each chunked column one thread that adds its chunk sums (the chunk
// launch ran before) in chunk order, as the CSR kernel does.  EPI (plain
// iterations): the thread that owns a column runs the primal update on it
// (operands loaded before the sum) instead of storing g for the elementwise
// launch; g is rounded as it would have been stored, so the iterates are
// bit-identical to the two-launch form that check iterations keep.  Blocks
// of two warps (the reason is the fused dual step's; 13k-bus LP: 0.1443 ms
// per primal step against 0.1461 ms with 256-thread blocks).
constexpr int kPrimalBlock = 64, kPrimalWpb = kPrimalBlock / 32;
template <int PREC, bool EPI>
__global__ void __launch_bounds__(kPrimalBlock, kDualMinBlocks * kBlock / kPrimalBlock) k_primal_sell(DevLP L, int j) {
  const Ctrl* ctrl = L.ctrl;
  if (ctrl->done) return;
  const bool fp64 = phase64(ctrl, PREC);
  PrimalEpi<false> epi{L, ctrl->sigma, EPI ? L.coef[2 * j] : 0.0, EPI ? L.coef[2 * j + 1] : 0.0, fp64,
                       ctrl->algo == SCUC_ALGO_PDHG_AVG, false, {0.0, 0.0, 0.0, 0.0}, 0.0, 0.0, 0.0, 0.0, 0.0};
  const int nsb = (L.sT.nslice + kPrimalWpb - 1) / kPrimalWpb;
  if ((int)blockIdx.x < nsb) {
    const int sl = (int)blockIdx.x * kPrimalWpb + (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (sl >= L.sT.nslice) return;
    if (!fp64) {
      int r;
      const float a = sell_sum32(L.sT, L.y32, sl, lane, r);
      if (EPI && r >= 0) epi.load(r);
      if (r >= 0) {
        if (EPI) epi.row(r, (double)a);
        else L.gsum32[r] = a;
      }
    } else {
      const int r = L.sT.rows[(size_t)sl * 32 + lane];
      const double a = sell_sum(L.sT, L.y, sl, lane);
      if (EPI && r >= 0) epi.load(r);
      if (r >= 0) {
        if (EPI) epi.row(r, a);
        else L.gsum[r] = a;
      }
    }
    return;
  }
  const int i = ((int)blockIdx.x - nsb) * kPrimalBlock + (int)threadIdx.x;
  if (i >= L.pT.nlong) return;
  const int r = L.pT.long_rows[i];
  if (EPI) epi.load(r);
  const double s = chunk_total(L.pT, i);
  if (EPI) epi.row(r, fp64 ? s : (double)(float)s);
  else if (!fp64) L.gsum32[r] = (float)s;
  else L.gsum[r] = s;
}

// Primal step, elementwise over the columns of LP blockIdx.y (blockIdx.x of
// epi_gx blocks strides over them): contiguous loads, full warps for the
// FP64 arithmetic.
template <bool CHECK, int PREC>
__global__ void __launch_bounds__(kBlock) k_primal_epi(DevLP L, int j) {
  const int lp = blockIdx.y;
  const Ctrl* ctrl = L.ctrl + lp;
  if (ctrl->done) return;
  const double* cf = L.coef + (size_t)lp * L.coef_stride;
  PrimalEpi<CHECK> epi{L, ctrl->sigma, cf[2 * j], cf[2 * j + 1], phase64(ctrl, PREC), ctrl->algo == SCUC_ALGO_PDHG_AVG,
                       ctrl->infeas_tol > 0.0, {0.0, 0.0, 0.0, 0.0}, 0.0, 0.0, 0.0, 0.0, 0.0};
  const float* g32 = L.gsum32;
  int c0, c1;
  lp_range(L.col0, lp, L.n, c0, c1);
  const int stride = gridDim.x * kBlock;
  for (int c = c0 + (int)blockIdx.x * kBlock + (int)threadIdx.x; c < c1; c += stride) {
    epi.load(c);
    epi.row(c, epi.fp64 ? L.gsum[c] : (double)g32[c]);
  }
  if (CHECK) block_store_slot<4>(epi.acc, L.partP, L.epi_gx * L.nlp, lp * L.epi_gx + (int)blockIdx.x);
}

// ---------------------------------------------------------------------------
// dual step over A x_t: y_bar = P_s(y - s A x_t), Halpern
// P_s(r) = r + s Pi_[lo,hi](-r/s) = max(r + s lo, 0) + min(r + s hi, 0)
// ---------------------------------------------------------------------------
template <bool CHECK>
struct DualEpi {
  const DevLP& L;
  double s, wa, wb;
  bool fp64;
  bool pdhg;  // y^{k+1} = y_bar, running average in ybar
  double acc[2];
  double yi, loi, hii, y0i;  // the row's operands, loaded before its sum
  __device__ void load(int i) {
    yi = L.y[i];
    loi = L.lo[i];
    hii = L.hi[i];
    y0i = L.y0[i];
  }
  __device__ void row(int i, double q) {
    const double r = yi - s * q;
    const double yb = max0(r + s * loi) + min0(r + s * hii);
    double yn, ya = 0.0;
    if (pdhg) {
      yn = yb;
      ya = wb == 0.0 ? yb : __dadd_rn(__dmul_rn(wa, yb), __dmul_rn(wb, L.ybar[i]));
      L.ybar[i] = ya;
    } else {
      yn = wa * y0i + wb * (2.0 * yb - yi);
    }
    L.y[i] = yn;
    if (!fp64) L.y32[i] = (float)yn;
    if (CHECK) {
      if (!pdhg) L.ybar[i] = yb;
      L.qchk[i] = q;
      L.dychk[i] = yb - yi;
      acc[0] += (yb - yi) * (yb - yi);
      const double d = (pdhg ? ya : yn) - y0i;
      acc[1] += d * d;
    }
  }
};

template <bool CHECK, int PREC>
__global__ void __launch_bounds__(kBlock, kDualMinBlocks) k_dual(DevLP L, int j) {
  extern __shared__ __align__(128) unsigned char smem[];
  const BlockPlan bp = spmv_plan<true>(L.pA);  // issued together with the control loads
  const int lp = L.blkA ? L.blkA[blockIdx.x] : 0;
  const Ctrl* ctrl = L.ctrl + lp;
  if (ctrl->done) return;
  const double* cf = L.coef + (size_t)lp * L.coef_stride;
  DualEpi<CHECK> epi{L, ctrl->s_step, cf[2 * j], cf[2 * j + 1], phase64(ctrl, PREC),
                     ctrl->algo == SCUC_ALGO_PDHG_AVG, {0.0, 0.0}, 0.0, 0.0, 0.0, 0.0};
  if (bp.er >= 0) epi.load(bp.er);
  if (epi.fp64) {
    spmv_run<double>(bp, L.rp, L.col, L.vs, L.xt, L.pA, smem, epi);
  } else {
    struct Wrap {
      DualEpi<CHECK>& e;
      __device__ void load(int r) { e.load(r); }
      __device__ void row(int r, float a) { e.row(r, (double)a); }
    } w{epi};
    spmv_run<float>(bp, L.rp, L.col, L.vs32, L.xt32, L.pA, smem, w);
  }
  if (CHECK) block_store<2>(epi.acc, L.partD, L.pA);
}

// Dual step of a plain iteration of one LP whose A has chunked long rows,
// in two launches: k_dual_fused runs the chunk warps of the long rows and
// the other rows on the sliced ELL copy of A (one warp per slice of 32 rows,
// the row's update in the lane that summed it: no shared memory, so the
// chunk warps' gathers keep the whole L1), interleaved evenly in one grid
// (block b is a slice block when floor((b + 1) ns / nb) > floor(b ns / nb)),
// so that warps streaming the long rows and warps running the short rows'
// FP64 updates share every SM; k_dual_long then adds each long row's chunk
// sums and runs its update.  Check iterations keep the chunk launch +
// k_dual form (its block partials feed the check).  Blocks of two warps: an
// SM gets a block's registers back only when its last warp has ended, so
// small blocks leave fewer finished warps' registers idle at the same
// occupancy (24 blocks of 64 threads per SM at 40 registers; on the 13k-bus
// LP 0.1611 ms per dual step against 0.1622 ms with 256-thread blocks).
constexpr int kDualBlock = 64, kDualWpb = kDualBlock / 32;
template <int PREC>
__global__ void __launch_bounds__(kDualBlock, kDualMinBlocks * kBlock / kDualBlock) k_dual_fused(DevLP L, int j) {
  const int ns = (L.sA.nslice + kDualWpb - 1) / kDualWpb;
  const int nb = ns + (L.pA.nchunk + kDualWpb - 1) / kDualWpb;
  const int b = (int)blockIdx.x;
  const int sb = (int)((int64_t)b * ns / nb);  // slice blocks before this one
  const bool slices = (int64_t)(b + 1) * ns / nb > sb;
  const Ctrl* ctrl = L.ctrl;
  if (ctrl->done) return;
  const bool fp64 = phase64(ctrl, PREC);
  if (!slices) {
    if (fp64) chunk_warp<double, kDualWpb>(L.col, L.vs, L.xt, L.pA, b - sb);
    else chunk_warp<float, kDualWpb>(L.col, L.vs32, L.xt32, L.pA, b - sb);
    return;
  }
  const int sl = sb * kDualWpb + (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (sl >= L.sA.nslice) return;
  DualEpi<false> epi{L, ctrl->s_step, L.coef[2 * j], L.coef[2 * j + 1], fp64, ctrl->algo == SCUC_ALGO_PDHG_AVG,
                     {0.0, 0.0}, 0.0, 0.0, 0.0, 0.0};
  if (!fp64) {
    int r;
    const float a = sell_sum32(L.sA, L.xt32, sl, lane, r);
    if (r >= 0) {
      epi.load(r);
      epi.row(r, (double)a);
    }
  } else {
    const int r = L.sA.rows[(size_t)sl * 32 + lane];
    const double a = sell_sum(L.sA, L.xt, sl, lane);
    if (r >= 0) {
      epi.load(r);
      epi.row(r, a);
    }
  }
}

// The long rows' updates after k_dual_fused: one thread per long row adds
// the row's chunk sums in chunk order (as the main launch's long-row blocks
// do), in blocks of 64 threads so that the few long rows spread over many
// SMs (the launch is a chain of dependent loads, not a stream).
template <int PREC>
__global__ void __launch_bounds__(64) k_dual_long(DevLP L, int j) {
  const Partition& P = L.pA;
  const int li = (int)blockIdx.x * 64 + (int)threadIdx.x;
  const int r = li < P.nlong ? P.long_rows[li] : -1;
  const Ctrl* ctrl = L.ctrl;
  if (ctrl->done || r < 0) return;
  DualEpi<false> epi{L, ctrl->s_step, L.coef[2 * j], L.coef[2 * j + 1], phase64(ctrl, PREC),
                     ctrl->algo == SCUC_ALGO_PDHG_AVG, {0.0, 0.0}, 0.0, 0.0, 0.0, 0.0};
  epi.load(r);
  const double t = chunk_total16(P, li);
  epi.row(r, epi.fp64 ? t : (double)(float)t);
}

// ---------------------------------------------------------------------------
// KKT check SpMVs (always FP64)
// ---------------------------------------------------------------------------
struct ResPrimalEpi {  // A x_bar: primal violation (unscaled), y-part of dobj, <A dx, dy>
  const DevLP& L;
  double beta;
  double acc[3];
  __device__ void load(int) {}
  __device__ void row(int i, double a) {
    const double lo = L.lo[i], hi = L.hi[i];
    const double viol = (a - clampd(a, lo, hi)) * beta / L.Dr[i];
    acc[0] += viol * viol;
    const double yb = L.ybar[i];
    if (yb > 0.0 && isfinite(lo)) acc[1] += lo * yb;
    else if (yb < 0.0 && isfinite(hi)) acc[1] += hi * yb;
    acc[2] += (L.qchk[i] - a) * L.dychk[i];   // A(x_bar - x) = A x_t - A x_bar
  }
};

__global__ void __launch_bounds__(kBlock) k_res_primal(DevLP L) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Ctrl* ctrl = L.ctrl + (L.blkA ? L.blkA[blockIdx.x] : 0);
  if (ctrl->done) return;
  ResPrimalEpi epi{L, ctrl->beta, {0.0, 0.0, 0.0}};
  spmv_block<double>(L.rp, L.col, L.vs, L.xbar, L.pA, smem, epi);
  block_store<3>(epi.acc, L.partRA, L.pA);
}

// A^T y_bar: dual residual (unscaled).  AVG (restarted PDHG): y_bar is the
// running average and z the reduced cost c - A^T y_bar where a finite bound
// lets it act (0 elsewhere), stored in zbar; acc[1] is its part of the dual
// objective (scaled).
template <bool AVG>
struct ResDualEpi {
  const DevLP& L;
  double gamma;
  double acc[AVG ? 2 : 1];
  __device__ void load(int) {}
  __device__ void row(int j, double g) {
    double z;
    if (AVG) {
      const double xl = L.xl[j], xu = L.xu[j];
      z = L.c[j] - g;
      if (z > 0.0 && !isfinite(xl)) z = 0.0;
      if (z < 0.0 && !isfinite(xu)) z = 0.0;
      L.zbar[j] = z;
      if (z > 0.0) acc[AVG ? 1 : 0] += xl * z;
      else if (z < 0.0) acc[AVG ? 1 : 0] += xu * z;
    } else {
      z = L.zbar[j];
    }
    const double d = gamma * (L.c[j] - g - z) / L.Dc[j];
    acc[0] += d * d;
  }
};

template <bool AVG>
__global__ void __launch_bounds__(kBlock) k_res_dual(DevLP L) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Ctrl* ctrl = L.ctrl + (L.blkT ? L.blkT[blockIdx.x] : 0);
  if (ctrl->done) return;
  ResDualEpi<AVG> epi{L, ctrl->gamma, {}};
  spmv_block<double>(L.rpt, L.colt, L.vst, L.ybar, L.pT, smem, epi);
  block_store<AVG ? 2 : 1>(epi.acc, L.partRT, L.pT);
}

// A^T v on the sliced copy of A^T with a per-column epilogue, for launches
// whose block partial sums the host or the decide kernel reads as nslot
// (= A^T's CSR partition block count) slots.  The grid has G = min(nslot,
// sell_blocks) blocks: block b takes slice blocks b, b + G, ... (8 slices
// each, one per warp) and long columns b * kBlock + t, (b + G) * kBlock + t,
// ... (their chunk sums already computed, added in chunk order), stores its
// Q partial sums in slot b and zeros in slots b + G, b + 2G, ... < nslot.
// Deterministic: fixed assignment, fixed orders.  VT: the product's value
// type (FP32 values: the FP32 form the copy holds).
__host__ __device__ inline int sell_blocks(const Sell& S, const Partition& pT) {
  return (S.nslice + kBlock / 32 - 1) / (kBlock / 32) + (pT.nlong + kBlock - 1) / kBlock;
}

template <int Q>
__device__ __forceinline__ void sell_store(const double (&v)[Q], double* out, int nslot) {
  block_store_slot<Q>(v, out, nslot, (int)blockIdx.x);
  for (int z = (int)(blockIdx.x + gridDim.x); z < nslot; z += (int)gridDim.x)
    if ((int)threadIdx.x < Q) out[threadIdx.x * nslot + z] = 0.0;
}

template <typename VT, class Epi>
__device__ __forceinline__ void sell_gridstride(const Sell& S, const Partition& pT, const VT* __restrict__ x,
                                                Epi& epi) {
  const int nslot = (int)gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nsb = (S.nslice + kBlock / 32 - 1) / (kBlock / 32);
  for (int sb = (int)blockIdx.x; sb < nsb; sb += nslot) {
    const int sl = sb * (kBlock / 32) + warp;
    if (sl >= S.nslice) continue;  // warp-uniform
    int r;
    VT a;
    if constexpr (sizeof(VT) == 4) {
      a = sell_sum32(S, x, sl, lane, r);
    } else {
      r = S.rows[(size_t)sl * 32 + lane];
      a = sell_sum(S, x, sl, lane);
    }
    if (r >= 0) epi.row(r, a);
  }
  for (int i = (int)blockIdx.x * kBlock + (int)threadIdx.x; i < pT.nlong; i += nslot * kBlock)
    epi.row(pT.long_rows[i], (VT)chunk_total(pT, i));
}

// Check iterations of one LP with a sliced copy of A^T: A^T y_bar and the
// dual residual (k_res_dual's epilogue and partial-sum slots).
template <bool AVG>
__global__ void __launch_bounds__(kBlock) k_res_dual_sell(DevLP L) {
  const Ctrl* ctrl = L.ctrl;
  if (ctrl->done) return;
  ResDualEpi<AVG> epi{L, ctrl->gamma, {}};
  sell_gridstride<double>(L.sT, L.pT, L.ybar, epi);
  sell_store<AVG ? 2 : 1>(epi.acc, L.partRT, L.pT.nblk);
}

// ---------------------------------------------------------------------------
// Infeasibility certificates at a check (scaled LP; scaling maps certificates
// to certificates).  Rays: u = y_bar - y (dychk) and d = x_bar - x (dxchk).
//  primal infeasible: F(u) = sum_i (u_i > 0 ? lo_i : hi_i) u_i
//    + sum_j (z_j > 0 ? xl_j : xu_j) z_j with z = -A^T u, over the terms whose
//    bound is finite, > 0; the other terms' squares are the violation;
//  unbounded: c^T d < 0 with A d and d in the recession cones of [lo, hi]
//    and [xl, xu]; the squares of the components outside are the violation.
// Rows (A d, u):   partRA slots 3, 4, 5 = cone violation of A d, F rows, violation rows.
// Columns (A^T u, d): partRT slots 2, 3, 4, 5 = F cols, violation cols, c^T d, cone violation of d.
// ---------------------------------------------------------------------------
struct InfRowsEpi {
  const DevLP& L;
  double acc[3];
  __device__ void load(int) {}
  __device__ void row(int i, double ad) {
    const double lo = L.lo[i], hi = L.hi[i], u = L.dychk[i];
    if ((ad < 0.0 && isfinite(lo)) || (ad > 0.0 && isfinite(hi))) acc[0] += ad * ad;
    if (u > 0.0) {
      if (isfinite(lo)) acc[1] += lo * u;
      else acc[2] += u * u;
    } else if (u < 0.0) {
      if (isfinite(hi)) acc[1] += hi * u;
      else acc[2] += u * u;
    }
  }
};

__global__ void __launch_bounds__(kBlock) k_inf_rows(DevLP L) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Ctrl* ctrl = L.ctrl + (L.blkA ? L.blkA[blockIdx.x] : 0);
  if (ctrl->done) return;
  InfRowsEpi epi{L, {0.0, 0.0, 0.0}};
  spmv_block<double>(L.rp, L.col, L.vs, L.dxchk, L.pA, smem, epi);
  block_store<3>(epi.acc, L.partRA + 3 * (size_t)L.pA.nblk, L.pA);
}

struct InfColsEpi {
  const DevLP& L;
  double acc[4];
  __device__ void load(int) {}
  __device__ void row(int j, double atu) {
    const double xl = L.xl[j], xu = L.xu[j], z = -atu, d = L.dxchk[j];
    if (z > 0.0) {
      if (isfinite(xl)) acc[0] += xl * z;
      else acc[1] += z * z;
    } else if (z < 0.0) {
      if (isfinite(xu)) acc[0] += xu * z;
      else acc[1] += z * z;
    }
    acc[2] += L.c[j] * d;
    if ((d < 0.0 && isfinite(xl)) || (d > 0.0 && isfinite(xu))) acc[3] += d * d;
  }
};

__global__ void __launch_bounds__(kBlock) k_inf_cols(DevLP L) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Ctrl* ctrl = L.ctrl + (L.blkT ? L.blkT[blockIdx.x] : 0);
  if (ctrl->done) return;
  InfColsEpi epi{L, {0.0, 0.0, 0.0, 0.0}};
  spmv_block<double>(L.rpt, L.colt, L.vst, L.dychk, L.pT, smem, epi);
  block_store<4>(epi.acc, L.partRT + 2 * (size_t)L.pT.nblk, L.pT);
}

// fixed-order sum of one partial array by a single block
__device__ double decide_sum(const double* p, int cnt) {
  double s = 0.0;
  for (int i = threadIdx.x; i < cnt; i += kDecideThreads) s += p[i];
  __shared__ double sm[kDecideThreads / 32];
  s = warp_sum(s);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kDecideThreads / 32; w++) r += sm[w];
  return r;
}

// ---------------------------------------------------------------------------
// decide: residuals, restart rule, sigma update, stop (one block)
// ---------------------------------------------------------------------------
// sums of the infeasibility certificates (k_inf_rows / k_inf_cols)
struct InfSums {
  double f, v;       // primal infeasibility: objective of the ray, squared violation
  double cd, vd;     // unboundedness: c^T d, squared cone violation
};

__device__ long long decide_logic(const DevLP& L, Ctrl* C, scuc_check_log* log, int chunk, double Sx,
                                  double Sxa, double pobj_s, double dz, double Sy, double Sya, double viol2,
                                  double dy, double dres2, double cross, const InfSums& inf);

// one block per LP of the batch (blockIdx.x = LP)
__global__ void __launch_bounds__(kDecideThreads) k_decide(DevLP L, int chunk) {
  const int lp = blockIdx.x;
  Ctrl* C = L.ctrl + lp;
  if (C->done) return;
  const int nA = L.pA.nblk, nT = L.pT.nblk, nP = L.epi_gx * L.nlp, p0 = lp * L.epi_gx;
  int a0, a1, t0, t1;
  lp_range(L.ablk0, lp, nA, a0, a1);
  lp_range(L.tblk0, lp, nT, t0, t1);
  const int ca = a1 - a0, ct = t1 - t0;
  const double Sx = decide_sum(L.partP + 0 * nP + p0, L.epi_gx);
  const double Sxa = decide_sum(L.partP + 1 * nP + p0, L.epi_gx);
  const double pobj_s = decide_sum(L.partP + 2 * nP + p0, L.epi_gx);
  const bool avg = C->algo == SCUC_ALGO_PDHG_AVG;  // z and its objective part come with A^T y_avg
  const double dz = avg ? decide_sum(L.partRT + 1 * nT + t0, ct) : decide_sum(L.partP + 3 * nP + p0, L.epi_gx);
  const double Sy = decide_sum(L.partD + 0 * nA + a0, ca);
  const double Sya = decide_sum(L.partD + 1 * nA + a0, ca);
  const double viol2 = decide_sum(L.partRA + 0 * nA + a0, ca);
  const double dy = decide_sum(L.partRA + 1 * nA + a0, ca);
  const double dres2 = decide_sum(L.partRT + t0, ct);
  const double cross = decide_sum(L.partRA + 2 * nA + a0, ca);
  InfSums inf{0.0, 0.0, 0.0, 0.0};
  if (C->infeas_tol > 0.0) {
    const double vq = decide_sum(L.partRA + 3 * nA + a0, ca);
    const double fr = decide_sum(L.partRA + 4 * nA + a0, ca);
    const double vr = decide_sum(L.partRA + 5 * nA + a0, ca);
    const double fc = decide_sum(L.partRT + 2 * nT + t0, ct);
    const double vc = decide_sum(L.partRT + 3 * nT + t0, ct);
    const double cd = decide_sum(L.partRT + 4 * nT + t0, ct);
    const double vd = decide_sum(L.partRT + 5 * nT + t0, ct);
    inf = InfSums{fr + fc, vr + vc, cd, vd + vq};
  }
  __shared__ long long s_knew;
  if (threadIdx.x == 0)
    s_knew = decide_logic(L, C, L.log + (size_t)lp * L.log_stride, chunk, Sx, Sxa, pobj_s, dz, Sy, Sya, viol2,
                          dy, dres2, cross, inf);
  __syncthreads();
  // weights of the next period, computed once (FP64 division is slow on this
  // part; every iterate update would otherwise divide per thread): Halpern
  // {1/(k+2), (k+1)/(k+2)}, or the running average's {1/(k+1), k/(k+1)}
  const long long kn = s_knew;
  double* cw = L.coef_w + (size_t)lp * L.coef_stride;
  for (int j = threadIdx.x; j < chunk; j += kDecideThreads) {
    if (avg) {
      cw[2 * j] = 1.0 / (double)(kn + j + 1);
      cw[2 * j + 1] = (double)(kn + j) / (double)(kn + j + 1);
    } else {
      cw[2 * j] = 1.0 / (double)(kn + j + 2);
      cw[2 * j + 1] = (double)(kn + j + 1) / (double)(kn + j + 2);
    }
  }
}

__device__ long long decide_logic(const DevLP& L, Ctrl* C, scuc_check_log* log, int chunk, double Sx,
                                  double Sxa, double pobj_s, double dz, double Sy, double Sya, double viol2,
                                  double dy, double dres2, double cross, const InfSums& inf) {

  const double sigma = C->sigma, lambda = C->lambda, bg = C->beta * C->gamma;
  const double rp = sqrt(viol2) / (1.0 + C->bnorm);
  const double rd = sqrt(dres2) / (1.0 + C->cnorm);
  const double pobj = bg * pobj_s, dobj = bg * (dy + dz);
  const double gap = fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
  // fmax returns its other operand for a NaN, so a NaN residual is carried
  // into kkt explicitly (it then stops the solve as SCUC_ST_NUMERICAL)
  const double kkt = (rp != rp || rd != rd || gap != gap) ? (double)NAN : fmax(rp, fmax(rd, gap));
  const int64_t k = C->k + chunk, t = C->t + chunk;
  const double rho = (C->restart_metric == 2 || C->algo == SCUC_ALGO_PDHG_AVG)
                         ? kkt
                         : sqrt(fmax(0.0, Sx / sigma + lambda * sigma * Sy +
                                              (C->restart_metric == 1 ? 2.0 * cross : 0.0)));
  C->rp = rp; C->rd = rd; C->gap = gap; C->pobj = pobj; C->dobj = dobj; C->kkt = kkt;
  if (!C->fp64_phase) C->iters_fp32 += chunk;

  int restart = 0, status = -1;
  const int was_first = C->first_check;
  if (!(kkt == kkt) || isinf(kkt)) {
    status = SCUC_ST_NUMERICAL;
  } else if (kkt <= C->tol) {
    status = SCUC_ST_OPTIMAL;
  } else if (C->infeas_tol > 0.0 && inf.f > 0.0 && sqrt(inf.v) <= C->infeas_tol * inf.f) {
    status = SCUC_ST_PRIMAL_INFEASIBLE;  // y_bar - y is a Farkas ray
  } else if (C->infeas_tol > 0.0 && inf.cd < 0.0 && sqrt(inf.vd) <= C->infeas_tol * -inf.cd) {
    status = SCUC_ST_DUAL_INFEASIBLE;    // x_bar - x is a direction of unbounded descent
  } else if (C->reject_kkt > 0.0 && t == (int64_t)C->check_every && kkt >= C->reject_kkt) {
    status = SCUC_ST_FALLBACK_COLD;  // a warm start whose first check is no better than the cold start
  } else {
    if (C->first_check) {
      C->rho0 = rho;
      C->first_check = 0;
      if ((double)k >= C->restart_long * (double)t) restart = 1;
    } else {
      if (rho <= C->restart_suff * C->rho0) restart = 1;
      else if (rho <= C->restart_nec * C->rho0 && rho > C->rho_prev) restart = 1;
      else if ((double)k >= C->restart_long * (double)t) restart = 1;
    }
    C->rho_prev = rho;
  }
  if (C->nlog < C->log_cap) {
    scuc_check_log& e = log[C->nlog];
    e.iter = t; e.restart = restart; e.first = was_first;
    e.rp = rp; e.rd = rd; e.gap = gap; e.pobj = pobj; e.dobj = dobj; e.rho = rho;
    e.sigma = sigma; e.fp64 = C->fp64_phase; e.pad = 0;
  }
  C->nlog++;
  C->restart_pending = 0;
  if (status < 0 && restart) {
    const double ddx = sqrt(Sxa), ddy = sqrt(Sya);
    if (C->sigma_update && ddx > 1e-10 && ddy > 1e-10) {
      const double sig_new = ddx / (sqrt(lambda) * ddy);
      C->sigma = sqrt(sig_new * sigma);
    }
    C->restart_pending = 1;
    if (C->restart_ref == 1) C->rho0 = rho;  // decrease is measured from here
    else C->first_check = 1;
    C->restarts++;
  }
  // mixed precision: move to FP64 matvecs near the tolerance or on a stall
  if (status < 0 && C->precision == SCUC_MIXED && !C->fp64_phase) {
    if (kkt < 0.9 * C->best_kkt) { C->best_kkt = kkt; C->stall = 0; }
    else C->stall++;
    if (kkt <= fmax(C->polish_factor * C->tol, C->polish_floor) || C->stall >= C->polish_stall) C->fp64_phase = 1;
  }
  C->k = restart ? 0 : k;
  C->t = t;
  C->s_step = 1.0 / (C->lambda * C->sigma);
  if (status < 0 && t >= C->max_iter) status = SCUC_ST_ITER_LIMIT;
  if (status < 0 && C->time_limit_ns > 0 && globaltimer_ns() - C->t_start_ns > C->time_limit_ns)
    status = SCUC_ST_TIME_LIMIT;
  if (status >= 0) {
    C->status = status;
    C->done = 1;
  }
  return C->k;
}

// Conditions of a solve graph (one launch per solve): the loop continues
// while some LP has not stopped; the precision branch follows LP 0 (graphs of
// one LP).  One block, after the decide kernel.
__global__ void __launch_bounds__(kDecideThreads) k_loop_cond(DevLP L, cudaGraphConditionalHandle loop,
                                                             cudaGraphConditionalHandle phase, int set_phase) {
  __shared__ int s_any;
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  for (int lp = threadIdx.x; lp < L.nlp; lp += kDecideThreads)
    if (!L.ctrl[lp].done) atomicOr(&s_any, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    cudaGraphSetConditional(loop, s_any ? 1u : 0u);
    if (set_phase) cudaGraphSetConditional(phase, L.ctrl[0].fp64_phase ? 1u : 0u);
  }
}

// restart: anchor <- current point (runs at the start of each period);
// restarted PDHG moves the iterate to the cycle's average first;
// blockIdx.y = LP of the batch
__global__ void k_anchor(DevLP L) {
  const int lp = blockIdx.y;
  const Ctrl* C = L.ctrl + lp;
  if (C->done || !C->restart_pending) return;
  const bool avg = C->algo == SCUC_ALGO_PDHG_AVG;
  int a, b;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  lp_range(L.col0, lp, L.n, a, b);
  for (int64_t i = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += stride) {
    if (avg) {
      const double v = L.xbar[i];
      L.x[i] = v;
      L.x0[i] = v;
    } else {
      L.x0[i] = L.x[i];
    }
  }
  lp_range(L.row0, lp, L.m, a, b);
  for (int64_t i = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += stride) {
    if (avg) {
      const double v = L.ybar[i];
      L.y[i] = v;
      L.y0[i] = v;
      L.y32[i] = (float)v;
    } else {
      L.y0[i] = L.y[i];
    }
  }
}

}  // namespace

}  // namespace scuc
