// Logic-driven fixing (Round + Algorithm 1, Sec. 4.1) and the presolve of
// Algorithm 2 (Sec. 4.2): activity-based bound propagation and the reduced
// LP (fixed columns folded into the row bounds, redundant rows dropped).
//
// Row activities, candidate bounds and the folded row bounds use explicitly
// rounded FP64 operations (no contraction); a row of at most 32 entries is
// summed by one thread in entry order, a longer row by one warp in a fixed
// order (entry q of the row into lane q mod 32, each lane in entry order,
// lanes combined by halving 16, 8, 4, 2, 1), so propagated bounds and
// reduced-LP data are bit-identical run to run; min/max over a column's
// candidates is order-free.  Every fixing and presolve decision is made
// from those values.
#include <chrono>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "lp.h"
#include "spmv.cuh"

namespace scuc {
namespace {

constexpr int kThreads = 256;

// one thread per item: the grid covers every item (no cap)
int grid1(int64_t work) {
  const int64_t g = (work + kThreads - 1) / kThreads;
  return (int)(g < 1 ? 1 : g);
}

// Round(s, tau) of Sec. 4.1
__device__ __forceinline__ int round_tau(double s, double tau) {
  if (s >= 1.0 - tau) return 1;
  if (s >= 0.0 && s <= tau) return 0;
  return -1;
}

// Algorithm 1, one thread per generator: fixes (u, v, w)_t for t = t_first..T-1
// while the rounded values are confident and consistent with Eq. 1; writes
// fix_out (-1 = free) and sets xl = xu = value on the fixed columns.
__global__ void k_fix(int G, int T, const double* __restrict__ x, const int* __restrict__ ui,
                      const int* __restrict__ vi, const int* __restrict__ wi,
                      const int8_t* __restrict__ u_init, double tau, int t_first,
                      int8_t* __restrict__ fix_out, double* __restrict__ xl, double* __restrict__ xu,
                      unsigned long long* __restrict__ nfixed) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int64_t base = (int64_t)g * T;
  for (int t = 0; t < T; t++) {
    fix_out[3 * (base + t) + 0] = -1;
    fix_out[3 * (base + t) + 1] = -1;
    fix_out[3 * (base + t) + 2] = -1;
  }
  unsigned long long cnt = 0;
  for (int t = t_first; t < T; t++) {
    const int ut = round_tau(x[ui[base + t]], tau);
    const int up = t > 0 ? round_tau(x[ui[base + t - 1]], tau) : (int)u_init[g];
    const int vt = round_tau(x[vi[base + t]], tau);
    const int wt = round_tau(x[wi[base + t]], tau);
    if (ut == -1 || up == -1 || vt == -1 || wt == -1) break;
    if (ut - up == vt - wt && vt + wt <= 1) {
      fix_out[3 * (base + t) + 0] = (int8_t)ut;
      fix_out[3 * (base + t) + 1] = (int8_t)vt;
      fix_out[3 * (base + t) + 2] = (int8_t)wt;
      const int cu = ui[base + t], cv = vi[base + t], cw = wi[base + t];
      xl[cu] = xu[cu] = (double)ut;
      xl[cv] = xu[cv] = (double)vt;
      xl[cw] = xu[cw] = (double)wt;
      cnt++;
    } else {
      break;
    }
  }
  if (cnt) atomicAdd(nfixed, cnt);
}

constexpr int kWarps = kThreads / 32;

// one warp per item
int grid_w(int64_t work) {
  const int64_t g = (work + kWarps - 1) / kWarps;
  return (int)(g < 1 ? 1 : g);
}

// lane partials combined by halving (lane 0 holds the total)
__device__ __forceinline__ double lanes_total(double v) {
#pragma unroll
  for (int w = 16; w > 0; w >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, w));
  return v;
}

__device__ __forceinline__ int lanes_count(int c) { return __reduce_add_sync(0xffffffffu, c); }

// Sign and infinity tests on the bit pattern (integer pipe; B300's FP64 pipe
// bounds these kernels).  pos(a) == (a > 0) and inf(a) == isinf(a) for
// every non-NaN double (NaN values are rejected when an LP is created).
__device__ __forceinline__ bool pos(double a) { return __double_as_longlong(a) > 0; }
__device__ __forceinline__ bool inf(double a) {
  return ((unsigned long long)__double_as_longlong(a) << 1) == 0xFFE0000000000000ull;
}

// Rounding margin of the row-level skip of k_col_propagate (far above the
// few units of 2^-53 that the candidate's three roundings can cost).
constexpr double kSkipRel = 1e-13;

// Safe slack of one side of a row for that skip: a candidate bound from
// this side can tighten column j (coefficient a, bounds [l, u]) only if the
// slack (hi - min activity, or max activity - lo) is below |a| (u - l)
// exactly; slack_safe is the computed slack less a margin that covers the
// rounding of the candidate's computation, so slack_safe >= |a| c_j (c_j,
// column_skip_range below) proves that the computed candidate cannot move
// the bound.  +inf: the side implies no bound (infinite row bound, the
// other activity within the bound, or two or more infinite contributions);
// -inf: exactly one infinite contribution (only its column gets a bound;
// never skipped).
__device__ __forceinline__ double slack_safe(double bound, double act, int cinf, bool active) {
  if (!active || cinf >= 2) return INFINITY;
  if (cinf == 1) return -INFINITY;
  const double d = __dsub_rn(bound, act);
  return __dsub_rn(d, __dadd_rn(kSkipRel * (fabs(bound) + fabs(act) + fabs(d)), 1e-300));
}

// c_j of the skip test: (u - l) and the size of the bounds, inflated by the
// margin; +inf for a column with an infinite bound (never skipped).
__device__ __forceinline__ double column_skip_range(double l, double u) {
  if (inf(l) || inf(u)) return INFINITY;
  return __dadd_rn(__dmul_rn(__dsub_rn(u, l), 1.0 + kSkipRel),
                   __dadd_rn(kSkipRel * (fabs(l) + fabs(u)), 1e-300));
}

// Rows and columns of at most kShortItem entries (all but the dense network
// rows and the columns in them) take one thread each, their sums in entry
// order; longer ones one warp each (entry q in lane q mod 32, lanes combined
// by halving).  On B300 a warp instruction on the FP64 pipe costs its
// issue slot whatever the active lanes, so a warp per short item would pay
// the warp's reductions and its lane-0 tail for a handful of entries.
constexpr int kShortItem = 32;

// Item k of list (thread or warp per item): list index, lane, entry stride.
template <bool WARP>
struct Item {
  int k, lane;
  static constexpr int step = WARP ? 32 : 1;
  __device__ Item() {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    k = WARP ? (int)(t >> 5) : (int)t;
    lane = WARP ? (int)(threadIdx.x & 31) : 0;
  }
};

// whether any of entries [e0, e1) has flag[idx[e]] set (the whole warp's
// answer for WARP)
template <bool WARP>
__device__ __forceinline__ bool any_flagged(const int* __restrict__ idx, const uint8_t* __restrict__ flag, int e0,
                                            int e1, int lane) {
  bool any = false;
  if (WARP) {
    for (int b = e0; b < e1 && !any; b += 32) {
      const int e = b + lane;
      any = __any_sync(0xffffffffu, e < e1 && flag[idx[e]]);
    }
  } else {
    for (int e = e0; e < e1 && !any; e++) any = flag[idx[e]] != 0;
  }
  return any;
}

template <bool WARP>
__device__ __forceinline__ double item_total(double v) { return WARP ? lanes_total(v) : v; }
template <bool WARP>
__device__ __forceinline__ int item_count(int c) { return WARP ? lanes_count(c) : c; }

// Activity range of each row of list over the current bounds: finite parts
// (in the order above) plus the number of infinite contributions, and the
// rows' safe slacks for k_col_propagate's skip.  After the first pass a row
// is recomputed only when one of its columns changed bounds in the previous
// pass (chg); otherwise its activity range is the one already stored.
// dirty[i] records whether row i was recomputed.
template <bool WARP>
__global__ void __launch_bounds__(kThreads) k_row_activity(const int* __restrict__ list, int cnt,
                                                           const int* __restrict__ rp, const int* __restrict__ col,
                                                           const double* __restrict__ val,
                                                           const double* __restrict__ xl,
                                                           const double* __restrict__ xu, double* __restrict__ mn,
                                                           double* __restrict__ mx, int* __restrict__ cmn,
                                                           int* __restrict__ cmx, const double* __restrict__ lo,
                                                           const double* __restrict__ hi, double2* __restrict__ slk,
                                                           const uint8_t* __restrict__ chg,
                                                           uint8_t* __restrict__ dirty, int first) {
  const Item<WARP> it;
  if (it.k >= cnt) return;
  const int i = list[it.k], lane = it.lane;
  const int e0 = rp[i], e1 = rp[i + 1];
  if (!first) {
    const bool any = any_flagged<WARP>(col, chg, e0, e1, lane);
    if (lane == 0) dirty[i] = any ? 1 : 0;
    if (!any) return;
  }
  double a_mn = 0.0, a_mx = 0.0;
  int c_mn = 0, c_mx = 0;
  for (int e = e0 + lane; e < e1; e += it.step) {
    const double a = val[e];
    const int j = col[e];
    const bool ap = pos(a);
    const double lmin = ap ? xl[j] : xu[j];
    const double lmax = ap ? xu[j] : xl[j];
    if (inf(lmin)) c_mn++;
    else a_mn = __dadd_rn(a_mn, __dmul_rn(a, lmin));
    if (inf(lmax)) c_mx++;
    else a_mx = __dadd_rn(a_mx, __dmul_rn(a, lmax));
  }
  a_mn = item_total<WARP>(a_mn);
  a_mx = item_total<WARP>(a_mx);
  c_mn = item_count<WARP>(c_mn);
  c_mx = item_count<WARP>(c_mx);
  if (lane == 0) {
    mn[i] = a_mn;
    mx[i] = a_mx;
    cmn[i] = c_mn;
    cmx[i] = c_mx;
    const double hii = hi[i], loi = lo[i];
    // the same side tests as k_col_propagate's
    const bool hi_act = !inf(hii) && !(c_mx == 0 && a_mx <= hii);
    const bool lo_act = !inf(loi) && !(c_mn == 0 && a_mn >= loi);
    slk[i] = make_double2(slack_safe(hii, a_mn, c_mn, hi_act), slack_safe(a_mx, loi, c_mx, lo_act));
  }
}

// One Jacobi pass for each column of list (thread or warp per column, over
// its A^T entries): candidate bounds from every row that can bind, integer
// rounding, acceptance thresholds.  Only column j's own bounds are read and
// written by its thread or warp; row activities come from the previous
// kernel, so the pass is Jacobi.  A row whose maximum activity cannot
// exceed hi (minimum cannot fall below lo) implies no bound from that side
// and is skipped.  After the first pass a column whose own bounds did not
// change in the previous pass (chg) and none of whose rows were recomputed
// (dirty) would repeat the previous pass's candidates and decisions
// exactly, so it is skipped; chg[j] then records whether column j changed in
// this pass.
template <bool WARP>
__global__ void __launch_bounds__(kThreads) k_col_propagate(const int* __restrict__ list, int cnt,
                                                            const int* __restrict__ rpt, const int* __restrict__ colt,
                                                            const double* __restrict__ valt,
                                                            const double* __restrict__ lo,
                                                            const double* __restrict__ hi,
                                                            const double* __restrict__ mn,
                                                            const double* __restrict__ mx,
                                                            const int* __restrict__ cmn,
                                                            const int* __restrict__ cmx,
                                                            const double2* __restrict__ slk,
                                                            const uint8_t* __restrict__ is_int,
                                                            double* __restrict__ xl, double* __restrict__ xu,
                                                            int* __restrict__ flags,
                                                            const uint8_t* __restrict__ dirty,
                                                            uint8_t* __restrict__ chg, int first) {
  const Item<WARP> it;
  if (it.k >= cnt) return;
  const int j = list[it.k], lane = it.lane;
  const int e0 = rpt[j], e1 = rpt[j + 1];
  if (!first && !chg[j] && !any_flagged<WARP>(colt, dirty, e0, e1, lane)) return;  // chg[j] stays 0
  const double oxl = xl[j], oxu = xu[j];
  const double cj = column_skip_range(oxl, oxu);
  double nlo = oxl, nhi = oxu;
  for (int e = e0 + lane; e < e1; e += it.step) {
    const int i = colt[e];
    const double a = valt[e];
    // Row-level skip: a side whose safe slack is at least |a| c_j gives a
    // candidate that cannot move column j's bound (for a > 0 on the hi side
    // the computed b = (hi - (mn - a l)) / a is then >= u, for a < 0 it is
    // <= l; likewise on the lo side), so its computation is left out and
    // the bounds are exactly those of the full computation.  Rows that
    // cannot bind (most dense network rows) take only this test.
    const double2 sk = slk[i];
    const double need = __dmul_rn(fabs(a), cj);
    const bool hi_skip = sk.x >= need, lo_skip = sk.y >= need;
    if (hi_skip && lo_skip) continue;
    const bool ap = pos(a);
    const double lmin = ap ? oxl : oxu;
    const double lmax = ap ? oxu : oxl;
    const double hii = hi[i], loi = lo[i], mni = mn[i], mxi = mx[i];
    const int cmni = cmn[i], cmxi = cmx[i];
    // A candidate b = q / a replaces the running bound only if it is
    // strictly tighter, and that needs q below (or above) the exact product
    // bound * a (rounding is monotone and the bound is representable).  The
    // rounded product is within 2^-53 of the exact one (plus 2^-1074 when it
    // underflows), so a q beyond it by more than 1e-15 of its size plus
    // 1e-300 cannot tighten the bound: the (slow) FP64 division is skipped
    // and the result is unchanged.
    if (!hi_skip && !inf(hii) && !(cmxi == 0 && mxi <= hii)) {  // a x_j <= hi - (min activity of the rest)
      const bool ok = inf(lmin) ? (cmni == 1) : (cmni == 0);
      if (ok) {
        const double rest = inf(lmin) ? mni : __dsub_rn(mni, __dmul_rn(a, lmin));
        const double q = __dsub_rn(hii, rest);
        const double p = __dmul_rn(ap ? nhi : nlo, a);  // b < nhi (a > 0) or b > nlo (a < 0) needs q < p
        if (!(q > p + 1e-15 * fabs(p) + 1e-300)) {
          const double b = __ddiv_rn(q, a);
          if (ap) { if (b < nhi) nhi = b; }
          else { if (b > nlo) nlo = b; }
        }
      }
    }
    if (!lo_skip && !inf(loi) && !(cmni == 0 && mni >= loi)) {  // a x_j >= lo - (max activity of the rest)
      const bool ok = inf(lmax) ? (cmxi == 1) : (cmxi == 0);
      if (ok) {
        const double rest = inf(lmax) ? mxi : __dsub_rn(mxi, __dmul_rn(a, lmax));
        const double q = __dsub_rn(loi, rest);
        const double p = __dmul_rn(ap ? nlo : nhi, a);  // b > nlo (a > 0) or b < nhi (a < 0) needs q > p
        if (!(q < p - 1e-15 * fabs(p) - 1e-300)) {
          const double b = __ddiv_rn(q, a);
          if (ap) { if (b > nlo) nlo = b; }
          else { if (b < nhi) nhi = b; }
        }
      }
    }
  }
  if (WARP) {
    // min/max are order-free; lanes that kept the column's own bounds leave
    // nothing to combine, so the tree runs only when some lane moved one
    const bool moved = __any_sync(0xffffffffu, __double_as_longlong(nlo) != __double_as_longlong(oxl) ||
                                                   __double_as_longlong(nhi) != __double_as_longlong(oxu));
    if (moved) {
#pragma unroll
      for (int w = 16; w > 0; w >>= 1) {
        const double ol = __shfl_down_sync(0xffffffffu, nlo, w), oh = __shfl_down_sync(0xffffffffu, nhi, w);
        if (ol > nlo) nlo = ol;
        if (oh < nhi) nhi = oh;
      }
    }
    if (lane != 0) return;
  }
  double l = nlo, u = nhi, nxl = oxl, nxu = oxu;
  int changed = 0;
  if (is_int[j]) {
    if (!inf(u)) u = floor(__dadd_rn(u, 1e-6));
    if (!inf(l)) l = ceil(__dsub_rn(l, 1e-6));
    if (l > nxl) { nxl = l; changed = 1; }
    if (u < nxu) { nxu = u; changed = 1; }
  } else {
    const double tl = 1e-9 * fmax(1.0, !inf(oxl) ? fabs(oxl) : 1.0);
    const double tu = 1e-9 * fmax(1.0, !inf(oxu) ? fabs(oxu) : 1.0);
    if (l > __dadd_rn(oxl, tl)) { nxl = l; changed = 1; }
    if (u < __dsub_rn(oxu, tu)) { nxu = u; changed = 1; }
  }
  if (changed) {
    xl[j] = nxl;
    xu[j] = nxu;
    atomicOr(flags + 0, 1);
  }
  chg[j] = (uint8_t)changed;
  if (nxl > __dadd_rn(nxu, 1e-6)) atomicOr(flags + 1, 1);
}

// Reduced-LP rows of list (thread or warp per row): fixed columns folded
// into the row bounds, activity range over the free columns, redundancy
// test.
template <bool WARP>
__global__ void __launch_bounds__(kThreads) k_reduce_rows(const int* __restrict__ list, int cnt,
                                                          const int* __restrict__ rp, const int* __restrict__ col,
                                                          const double* __restrict__ val,
                                                          const double* __restrict__ lo,
                                                          const double* __restrict__ hi,
                                                          const double* __restrict__ xl,
                                                          const double* __restrict__ xu, int* __restrict__ keep,
                                                          int* __restrict__ knz, double* __restrict__ lo_r,
                                                          double* __restrict__ hi_r, int* __restrict__ flags) {
  const Item<WARP> it;
  if (it.k >= cnt) return;
  const int i = list[it.k], lane = it.lane;
  double shift = 0.0, a_mn = 0.0, a_mx = 0.0;
  int kept = 0, c_mn = 0, c_mx = 0;
  for (int e = rp[i] + lane; e < rp[i + 1]; e += it.step) {
    const int j = col[e];
    const double a = val[e], l = xl[j], u = xu[j];
    if (l == u) {
      shift = __dadd_rn(shift, __dmul_rn(a, l));
    } else {
      kept++;
      const bool ap = pos(a);
      const double lmin = ap ? l : u;
      const double lmax = ap ? u : l;
      if (inf(lmin)) c_mn++;
      else a_mn = __dadd_rn(a_mn, __dmul_rn(a, lmin));
      if (inf(lmax)) c_mx++;
      else a_mx = __dadd_rn(a_mx, __dmul_rn(a, lmax));
    }
  }
  shift = item_total<WARP>(shift);
  a_mn = item_total<WARP>(a_mn);
  a_mx = item_total<WARP>(a_mx);
  kept = item_count<WARP>(kept);
  c_mn = item_count<WARP>(c_mn);
  c_mx = item_count<WARP>(c_mx);
  if (lane != 0) return;
  const double l = __dsub_rn(lo[i], shift), u = __dsub_rn(hi[i], shift);
  lo_r[i] = l;
  hi_r[i] = u;
  if (kept == 0) {
    if (l > 1e-6 * fmax(1.0, fabs(l)) || u < -1e-6 * fmax(1.0, fabs(u))) atomicOr(flags + 1, 1);
    keep[i] = 0;
    knz[i] = 0;
    return;
  }
  const bool lo_red = inf(l) || (c_mn == 0 && a_mn >= l);
  const bool hi_red = inf(u) || (c_mx == 0 && a_mx <= u);
  keep[i] = (lo_red && hi_red) ? 0 : 1;
  knz[i] = keep[i] ? kept : 0;
}

// items (rows of a CSR) of at most kShortItem entries first, then the
// others, each group in index order: flag pass, then scatter by the scan
__global__ void k_short_flag(const int* __restrict__ rp, int m, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) flag[i] = rp[i + 1] - rp[i] <= kShortItem ? 1 : 0;
}

__global__ void k_split_list(int m, const int* __restrict__ flag, const int* __restrict__ pos, int nshort,
                             int* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  if (flag[i]) out[pos[i]] = i;
  else out[nshort + (i - pos[i])] = i;
}

__global__ void k_col_keep(int n, const double* __restrict__ xl, const double* __restrict__ xu,
                           int* __restrict__ keepc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) keepc[j] = xl[j] != xu[j] ? 1 : 0;
}

// kept rows: entries of free columns, renumbered, in the original order
// (warp per row; a ballot orders each 32-entry slice).  offs[i] is the first
// reduced entry of row i (exclusive scan of the kept counts); posr[e], when
// given, gets the reduced position of each copied entry e.
__global__ void __launch_bounds__(kThreads) k_scatter_rows(const int* __restrict__ rp, const int* __restrict__ col,
                                                           const double* __restrict__ val, int m,
                                                           const int* __restrict__ keep,
                                                           const int* __restrict__ newrow,
                                                           const int* __restrict__ offs,
                                                           const int* __restrict__ newcol,
                                                           const int* __restrict__ keepc,
                                                           const double* __restrict__ lo_t,
                                                           const double* __restrict__ hi_t, int* __restrict__ rp_r,
                                                           int* __restrict__ col_r, double* __restrict__ val_r,
                                                           double* __restrict__ lo_r, double* __restrict__ hi_r,
                                                           int* __restrict__ row_map, int* __restrict__ posr) {
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= m || !keep[i]) return;
  const int r = newrow[i];
  int k = offs[i];
  for (int e0 = rp[i]; e0 < rp[i + 1]; e0 += 32) {
    const int e = e0 + lane;
    const bool in = e < rp[i + 1];
    const int j = in ? col[e] : 0;
    const bool take = in && keepc[j];
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    if (take) {
      const int pos = k + __popc(bal & ((1u << lane) - 1u));
      col_r[pos] = newcol[j];
      val_r[pos] = val[e];
      if (posr) posr[e] = pos;
    }
    k += __popc(bal);
  }
  if (lane == 0) {
    rp_r[r] = offs[i];
    lo_r[r] = lo_t[i];
    hi_r[r] = hi_t[i];
    row_map[r] = i;
  }
}

// Reduced A^T from the parent's, which is sorted by row within each column:
// a kept column keeps its entries in kept rows, in the same order (newrow is
// increasing), so no sort is needed.  Warp per parent column.
__global__ void __launch_bounds__(kThreads) k_count_kept_t(const int* __restrict__ rpt, const int* __restrict__ colt,
                                                           int n, const int* __restrict__ keepc,
                                                           const int* __restrict__ newcol,
                                                           const int* __restrict__ keep, int* __restrict__ cnt) {
  const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (j >= n || !keepc[j]) return;
  int c = 0;
  for (int e = rpt[j] + lane; e < rpt[j + 1]; e += 32) c += keep[colt[e]] ? 1 : 0;
  c = __reduce_add_sync(0xffffffffu, c);
  if (lane == 0) cnt[newcol[j]] = c;
}

__global__ void __launch_bounds__(kThreads) k_compact_t(const int* __restrict__ rpt, const int* __restrict__ colt,
                                                        const int* __restrict__ permt,
                                                        const double* __restrict__ valt, int n,
                                                        const int* __restrict__ keepc,
                                                        const int* __restrict__ newcol,
                                                        const int* __restrict__ keep,
                                                        const int* __restrict__ newrow,
                                                        const int* __restrict__ posr,
                                                        const int* __restrict__ rpt_r, int* __restrict__ colt_r,
                                                        int* __restrict__ permt_r, double* __restrict__ valt_r) {
  const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (j >= n || !keepc[j]) return;
  int k = rpt_r[newcol[j]];
  for (int e0 = rpt[j]; e0 < rpt[j + 1]; e0 += 32) {
    const int e = e0 + lane;
    const bool in = e < rpt[j + 1];
    const int i = in ? colt[e] : 0;
    const bool take = in && keep[i];
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    if (take) {
      const int pos = k + __popc(bal & ((1u << lane) - 1u));
      colt_r[pos] = newrow[i];
      permt_r[pos] = posr[permt[e]];
      valt_r[pos] = valt[e];
    }
    k += __popc(bal);
  }
}

__global__ void k_scatter_cols(int n, const int* __restrict__ keepc, const int* __restrict__ newcol,
                               const double* __restrict__ c, const double* __restrict__ xl,
                               const double* __restrict__ xu, double* __restrict__ c_r,
                               double* __restrict__ xl_r, double* __restrict__ xu_r, int* __restrict__ col_map) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || !keepc[j]) return;
  const int k = newcol[j];
  c_r[k] = c[j];
  xl_r[k] = xl[j];
  xu_r[k] = xu[j];
  col_map[k] = j;
}

// objective of the fixed columns (one block, fixed order)
// objective of the fixed columns, sum_j c_j x_j over xl_j == xu_j: block b
// sums columns [b * per, (b + 1) * per) (thread-strided, then a fixed warp
// and block tree) into part[b]; k_sum_parts adds the blocks in order
constexpr int kObjBlocks = 296;
__global__ void __launch_bounds__(kThreads) k_fixed_obj(int n, const double* __restrict__ c,
                                                        const double* __restrict__ xl,
                                                        const double* __restrict__ xu, double* __restrict__ part) {
  __shared__ double s_w[kThreads / 32];
  const int per = (n + kObjBlocks - 1) / kObjBlocks;
  const int j0 = (int)blockIdx.x * per, j1 = min(n, j0 + per);
  double s = 0.0;
  for (int j = j0 + (int)threadIdx.x; j < j1; j += kThreads)
    if (xl[j] == xu[j]) s += c[j] * xl[j];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kThreads / 32; w++) r += s_w[w];
    part[blockIdx.x] = r;
  }
}

__global__ void k_sum_parts(const double* __restrict__ part, int k, double* __restrict__ out) {
  double r = 0.0;
  for (int b = 0; b < k; b++) r += part[b];
  *out = r;
}

}  // namespace

int Handle::build_fix_lists() {
  if (fix_lists) return SCUC_OK;
  cudaStream_t s = work;
  int* lists = nullptr;
  SCUC_TRY(alloc(&lists, (size_t)m + n + 1));
  void *fq = nullptr, *pq = nullptr;
  SCUC_TRY(dev_alloc_bytes(&fq, ((size_t)std::max(m, n) + 1) * sizeof(int)));
  struct Free {  // after the stream's work that uses them
    cudaStream_t s;
    void *a, *b;
    ~Free() {
      cudaStreamSynchronize(s);
      if (a) dev_free(a);
      if (b) dev_free(b);
    }
  } fr{s, fq, nullptr};
  SCUC_TRY(dev_alloc_bytes(&pq, ((size_t)std::max(m, n) + 1) * sizeof(int)));
  fr.b = pq;
  int *flag = static_cast<int*>(fq), *pos = static_cast<int*>(pq);
  int counts[2] = {0, 0};
  for (int t = 0; t < 2; t++) {
    const int k = t == 0 ? m : n;
    const int* ptr = t == 0 ? rp : rpt;
    if (k == 0) continue;
    k_short_flag<<<grid1(k), kThreads, 0, s>>>(ptr, k, flag);
    SCUC_TRY(exclusive_scan(flag, k, pos, s));
    SCUC_CUDA(cudaMemcpyAsync(&counts[t], pos + k, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaStreamSynchronize(s));
    k_split_list<<<grid1(k), kThreads, 0, s>>>(k, flag, pos, counts[t], lists + (t == 0 ? 0 : m));
    SCUC_CUDA(cudaGetLastError());
  }
  SCUC_CUDA(cudaStreamSynchronize(s));
  fix_lists = lists;
  fix_short_rows = counts[0];
  fix_short_cols = counts[1];
  return SCUC_OK;
}

int Handle::fix_and_propagate(const scuc_map& map, const uint8_t* is_int_h, const double* x_in,
                              const scuc_fix_params& p, int8_t* fix_out_h, Handle** reduced,
                              int32_t* col_map_h, int32_t* row_map_h, scuc_fix_info* info) {
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  if (map.G < 0 || map.T < 1 || (map.G > 0 && (!map.u_idx || !map.v_idx || !map.w_idx || !map.u_init)) ||
      !(p.tau >= 0.0 && p.tau < 0.5) || p.t_first < 0 || p.t_first > 1 || p.max_passes < 0 || !x_in) {
    set_error("scuc_fix_and_propagate: invalid map or parameters");
    return SCUC_E_INVALID;
  }
  const int64_t GT = (int64_t)map.G * map.T;
  for (int64_t k = 0; k < GT; k++) {
    const int32_t a = map.u_idx[k], b = map.v_idx[k], c2 = map.w_idx[k];
    if (a < 0 || a >= n || b < 0 || b >= n || c2 < 0 || c2 >= n) {
      set_error("scuc_fix_and_propagate: map index out of range at %lld", (long long)k);
      return SCUC_E_INVALID;
    }
  }
  SCUC_TRY(enter());
  SCUC_TRY(build_fix_lists());
  cudaStream_t s = work;
  std::vector<void*> tmp;
  auto talloc = [&](auto** ptr, size_t count) -> int {
    void* q = nullptr;
    SCUC_TRY(dev_alloc_bytes(&q, count * sizeof(**ptr)));
    tmp.push_back(q);
    *ptr = static_cast<std::remove_reference_t<decltype(*ptr)>>(q);
    return SCUC_OK;
  };
  struct Free {  // temporaries, after the stream's work that uses them
    cudaStream_t s;
    std::vector<void*>& v;
    ~Free() {
      if (!v.empty()) cudaStreamSynchronize(s);
      for (void* q : v) dev_free(q);
    }
  } freer{s, tmp};

  int *ui = nullptr, *vi = nullptr, *wi = nullptr, *flags = nullptr;
  int8_t *uinit = nullptr, *fixd = nullptr;
  uint8_t* isint = nullptr;
  unsigned long long* nfix = nullptr;
  double* xd = nullptr;
  SCUC_TRY(talloc(&ui, GT));
  SCUC_TRY(talloc(&vi, GT));
  SCUC_TRY(talloc(&wi, GT));
  SCUC_TRY(talloc(&uinit, map.G));
  SCUC_TRY(talloc(&fixd, 3 * GT));
  SCUC_TRY(talloc(&isint, n));
  SCUC_TRY(talloc(&flags, 2));
  SCUC_TRY(talloc(&nfix, 1));
  if (GT) {
    SCUC_CUDA(cudaMemcpyAsync(ui, map.u_idx, GT * sizeof(int), cudaMemcpyHostToDevice, s));
    SCUC_CUDA(cudaMemcpyAsync(vi, map.v_idx, GT * sizeof(int), cudaMemcpyHostToDevice, s));
    SCUC_CUDA(cudaMemcpyAsync(wi, map.w_idx, GT * sizeof(int), cudaMemcpyHostToDevice, s));
    SCUC_CUDA(cudaMemcpyAsync(uinit, map.u_init, map.G, cudaMemcpyHostToDevice, s));
  }
  std::vector<uint8_t> isint_h;
  if (!is_int_h) {  // default: the map's u, v, w columns
    isint_h.assign(n, 0);
    for (int64_t k = 0; k < GT; k++) isint_h[map.u_idx[k]] = isint_h[map.v_idx[k]] = isint_h[map.w_idx[k]] = 1;
    is_int_h = isint_h.data();
  }
  if (n) SCUC_CUDA(cudaMemcpyAsync(isint, is_int_h, n, cudaMemcpyHostToDevice, s));
  if (p.x_on_device) {
    xd = const_cast<double*>(x_in);
  } else {
    SCUC_TRY(talloc(&xd, n));
    SCUC_CUDA(cudaMemcpyAsync(xd, x_in, n * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  SCUC_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int), s));
  SCUC_CUDA(cudaMemsetAsync(nfix, 0, sizeof(unsigned long long), s));

  // F1/F2: Round + Algorithm 1, fixing the bounds of the model
  if (map.G > 0)
    k_fix<<<grid1(map.G), kThreads, 0, s>>>(map.G, map.T, xd, ui, vi, wi, uinit, p.tau, p.t_first, fixd, xl, xu,
                                            nfix);
  SCUC_CUDA(cudaGetLastError());

  // F3: Jacobi propagation
  double *mn = nullptr, *mx = nullptr;
  int *cmn = nullptr, *cmx = nullptr;
  uint8_t *chg = nullptr, *dirty = nullptr;
  double2* slk = nullptr;
  SCUC_TRY(talloc(&slk, m));
  SCUC_TRY(talloc(&mn, m));
  SCUC_TRY(talloc(&mx, m));
  SCUC_TRY(talloc(&cmn, m));
  SCUC_TRY(talloc(&cmx, m));
  SCUC_TRY(talloc(&chg, n));
  SCUC_TRY(talloc(&dirty, m));
  int passes = 0, infeasible = 0;
  int hflags[2] = {0, 0};
  const int *rows_s = fix_lists, *rows_l = fix_lists + fix_short_rows;
  const int *cols_s = fix_lists + m, *cols_l = fix_lists + m + fix_short_cols;
  const int nrs = fix_short_rows, nrl = m - fix_short_rows, ncs = fix_short_cols, ncl = n - fix_short_cols;
  for (int pass = 0; pass < p.max_passes; pass++) {
    SCUC_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), s));  // changed; flags[1] (infeasible) persists
    const int first = pass == 0 ? 1 : 0;
    if (nrl)
      k_row_activity<true><<<grid_w(nrl), kThreads, 0, s>>>(rows_l, nrl, rp, col, val, xl, xu, mn, mx, cmn, cmx,
                                                             lo, hi, slk, chg, dirty, first);
    if (nrs)
      k_row_activity<false><<<grid1(nrs), kThreads, 0, s>>>(rows_s, nrs, rp, col, val, xl, xu, mn, mx, cmn, cmx,
                                                             lo, hi, slk, chg, dirty, first);
    if (ncl)
      k_col_propagate<true><<<grid_w(ncl), kThreads, 0, s>>>(cols_l, ncl, rpt, colt, valt, lo, hi, mn, mx, cmn,
                                                              cmx, slk, isint, xl, xu, flags, dirty, chg, first);
    if (ncs)
      k_col_propagate<false><<<grid1(ncs), kThreads, 0, s>>>(cols_s, ncs, rpt, colt, valt, lo, hi, mn, mx, cmn,
                                                              cmx, slk, isint, xl, xu, flags, dirty, chg, first);
    SCUC_CUDA(cudaGetLastError());
    SCUC_CUDA(cudaMemcpyAsync(hflags, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaStreamSynchronize(s));
    passes = pass + 1;
    if (hflags[1]) { infeasible = 1; break; }
    if (!hflags[0]) break;
  }
  unsigned long long nf = 0;
  SCUC_CUDA(cudaMemcpyAsync(&nf, nfix, sizeof(nf), cudaMemcpyDeviceToHost, s));
  if (fix_out_h && GT) SCUC_CUDA(cudaMemcpyAsync(fix_out_h, fixd, 3 * GT, cudaMemcpyDeviceToHost, s));
  SCUC_CUDA(cudaStreamSynchronize(s));

  scuc_fix_info I{};
  const auto t_prop = clk::now();
  I.ms_propagate = std::chrono::duration<double, std::milli>(t_prop - t0).count();
  I.nfixed = (int64_t)nf;
  I.passes = passes;
  I.infeasible = infeasible;
  if (!infeasible && (reduced || col_map_h || row_map_h || info)) {
    // reduced LP
    int *keep = nullptr, *knz = nullptr, *keepc = nullptr, *newrow = nullptr, *newcol = nullptr, *offs = nullptr;
    double *lo_t = nullptr, *hi_t = nullptr, *objc = nullptr;
    SCUC_TRY(talloc(&keep, m + 1));
    SCUC_TRY(talloc(&knz, m + 1));
    SCUC_TRY(talloc(&keepc, n + 1));
    SCUC_TRY(talloc(&newrow, m + 1));
    SCUC_TRY(talloc(&newcol, n + 1));
    SCUC_TRY(talloc(&offs, m + 1));
    SCUC_TRY(talloc(&lo_t, m));
    SCUC_TRY(talloc(&hi_t, m));
    SCUC_TRY(talloc(&objc, 1 + kObjBlocks));
    if (nrl)
      k_reduce_rows<true><<<grid_w(nrl), kThreads, 0, s>>>(rows_l, nrl, rp, col, val, lo, hi, xl, xu, keep, knz,
                                                            lo_t, hi_t, flags);
    if (nrs)
      k_reduce_rows<false><<<grid1(nrs), kThreads, 0, s>>>(rows_s, nrs, rp, col, val, lo, hi, xl, xu, keep, knz,
                                                            lo_t, hi_t, flags);
    if (n) k_col_keep<<<grid1(n), kThreads, 0, s>>>(n, xl, xu, keepc);
    k_fixed_obj<<<kObjBlocks, kThreads, 0, s>>>(n, c, xl, xu, objc + 1);
    k_sum_parts<<<1, 1, 0, s>>>(objc + 1, kObjBlocks, objc);
    SCUC_CUDA(cudaGetLastError());
    SCUC_TRY(exclusive_scan(keep, m, newrow, s));   // reduced row of each kept row; newrow[m] = rows kept
    SCUC_TRY(exclusive_scan(keepc, n, newcol, s));  // reduced column of each free column
    SCUC_TRY(exclusive_scan(knz, m, offs, s));      // first reduced entry of each kept row; offs[m] = entries
    int mr = 0, nr = 0, nnzr = 0;
    SCUC_CUDA(cudaMemcpyAsync(&mr, newrow + m, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaMemcpyAsync(&nr, newcol + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaMemcpyAsync(&nnzr, offs + m, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaMemcpyAsync(hflags, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaMemcpyAsync(&I.obj_const, objc, sizeof(double), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaStreamSynchronize(s));
    I.infeasible = hflags[1] ? 1 : 0;
    I.n_fixed_cols = n - nr;
    I.m_red = mr;
    I.n_red = nr;
    I.nnz_red = nnzr;
    // device arrays of the reduced LP and its transpose (ownership passes to the new handle)
    void *d_rp = nullptr, *d_col = nullptr, *d_val = nullptr, *d_c = nullptr, *d_xl = nullptr, *d_xu = nullptr,
         *d_lo = nullptr, *d_hi = nullptr, *d_rpt = nullptr, *d_colt = nullptr, *d_permt = nullptr,
         *d_valt = nullptr;
    std::vector<void*> owned;
    struct FreeOwned {  // arrays not passed to the reduced handle, after the stream's work
      cudaStream_t s;
      std::vector<void*>& v;
      ~FreeOwned() {
        if (!v.empty()) cudaStreamSynchronize(s);
        for (void* q : v) dev_free(q);
      }
    } free_owned{s, owned};
    auto oalloc = [&](void** q, size_t bytes) -> int {
      SCUC_TRY(dev_alloc_bytes(q, bytes));
      owned.push_back(*q);
      return SCUC_OK;
    };
    SCUC_TRY(oalloc(&d_rp, (mr + 1) * sizeof(int)));
    SCUC_TRY(oalloc(&d_col, nnzr * sizeof(int)));
    SCUC_TRY(oalloc(&d_val, nnzr * sizeof(double)));
    SCUC_TRY(oalloc(&d_c, nr * sizeof(double)));
    SCUC_TRY(oalloc(&d_xl, nr * sizeof(double)));
    SCUC_TRY(oalloc(&d_xu, nr * sizeof(double)));
    SCUC_TRY(oalloc(&d_lo, mr * sizeof(double)));
    SCUC_TRY(oalloc(&d_hi, mr * sizeof(double)));
    const bool want_t = reduced && !I.infeasible;
    int *rmap = nullptr, *cmap = nullptr, *posr = nullptr, *cntr = nullptr;
    SCUC_TRY(talloc(&rmap, mr));
    SCUC_TRY(talloc(&cmap, nr));
    if (want_t) SCUC_TRY(talloc(&posr, nnz));
    int* rp_dev = static_cast<int*>(d_rp);
    if (m)
      k_scatter_rows<<<grid_w(m), kThreads, 0, s>>>(rp, col, val, m, keep, newrow, offs, newcol, keepc, lo_t, hi_t,
                                                   rp_dev, static_cast<int*>(d_col), static_cast<double*>(d_val),
                                                   static_cast<double*>(d_lo), static_cast<double*>(d_hi), rmap,
                                                   posr);
    SCUC_CUDA(cudaMemcpyAsync(rp_dev + mr, offs + m, sizeof(int), cudaMemcpyDeviceToDevice, s));
    if (n)
      k_scatter_cols<<<grid1(n), kThreads, 0, s>>>(n, keepc, newcol, c, xl, xu, static_cast<double*>(d_c),
                                                   static_cast<double*>(d_xl), static_cast<double*>(d_xu), cmap);
    SCUC_CUDA(cudaGetLastError());
    std::vector<int> rp_h, rpt_h;
    if (want_t) {
      SCUC_TRY(oalloc(&d_rpt, (nr + 1) * sizeof(int)));
      SCUC_TRY(oalloc(&d_colt, nnzr * sizeof(int)));
      SCUC_TRY(oalloc(&d_permt, nnzr * sizeof(int)));
      SCUC_TRY(oalloc(&d_valt, nnzr * sizeof(double)));
      SCUC_TRY(talloc(&cntr, nr + 1));
      int* rpt_r = static_cast<int*>(d_rpt);
      if (n) k_count_kept_t<<<grid_w(n), kThreads, 0, s>>>(rpt, colt, n, keepc, newcol, keep, cntr);
      SCUC_CUDA(cudaGetLastError());
      SCUC_TRY(exclusive_scan(cntr, nr, rpt_r, s));
      if (n)
        k_compact_t<<<grid_w(n), kThreads, 0, s>>>(rpt, colt, permt, valt, n, keepc, newcol, keep, newrow, posr,
                                                   rpt_r, static_cast<int*>(d_colt), static_cast<int*>(d_permt),
                                                   static_cast<double*>(d_valt));
      SCUC_CUDA(cudaGetLastError());
      rp_h.resize(mr + 1);
      rpt_h.resize(nr + 1);
      SCUC_CUDA(cudaMemcpyAsync(rp_h.data(), rp_dev, (mr + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
      SCUC_CUDA(cudaMemcpyAsync(rpt_h.data(), rpt_r, (nr + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    if (row_map_h && mr) SCUC_CUDA(cudaMemcpyAsync(row_map_h, rmap, mr * sizeof(int), cudaMemcpyDeviceToHost, s));
    if (col_map_h && nr) SCUC_CUDA(cudaMemcpyAsync(col_map_h, cmap, nr * sizeof(int), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaStreamSynchronize(s));
    const auto t_red = clk::now();
    I.ms_reduce = std::chrono::duration<double, std::milli>(t_red - t_prop).count();
    if (want_t) {
      owned.clear();  // the new handle frees them, also when its set-up fails
      Handle* H = new Handle();
      const DevTranspose T{static_cast<int*>(d_rpt), static_cast<int*>(d_colt), static_cast<int*>(d_permt),
                           static_cast<double*>(d_valt), &rp_h, &rpt_h};
      const int rc = H->init_device(mr, nr, nnzr, rp_dev, static_cast<int*>(d_col), static_cast<double*>(d_val),
                                    static_cast<double*>(d_c), static_cast<double*>(d_xl),
                                    static_cast<double*>(d_xu), static_cast<double*>(d_lo),
                                    static_cast<double*>(d_hi), user, &T);
      if (rc != SCUC_OK) {
        delete H;
        return rc;
      }
      *reduced = H;
      I.ms_setup = std::chrono::duration<double, std::milli>(clk::now() - t_red).count();
    }
  }
  I.ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
  if (info) *info = I;
  SCUC_TRY(leave());
  return I.infeasible ? SCUC_E_INFEASIBLE : SCUC_OK;
}

int Handle::get_bounds(double* xl_h, double* xu_h) {
  SCUC_TRY(enter());
  if (n && xl_h) SCUC_CUDA(cudaMemcpyAsync(xl_h, xl, n * sizeof(double), cudaMemcpyDeviceToHost, work));
  if (n && xu_h) SCUC_CUDA(cudaMemcpyAsync(xu_h, xu, n * sizeof(double), cudaMemcpyDeviceToHost, work));
  SCUC_CUDA(cudaStreamSynchronize(work));
  return leave();
}

int Handle::set_bounds(const double* xl_in, const double* xu_in, int on_device) {
  if (!on_device)
    for (int32_t j = 0; j < n; j++)
      if (std::isnan(xl_in[j]) || std::isnan(xu_in[j]) || xl_in[j] > xu_in[j] || xl_in[j] == INFINITY ||
          xu_in[j] == -INFINITY) {
        set_error("scuc_lp_set_bounds: invalid bounds at column %d", j);
        return SCUC_E_INVALID;
      }
  SCUC_TRY(enter());
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (n) {
    SCUC_CUDA(cudaMemcpyAsync(xl, xl_in, n * sizeof(double), k, work));
    SCUC_CUDA(cudaMemcpyAsync(xu, xu_in, n * sizeof(double), k, work));
  }
  SCUC_CUDA(cudaStreamSynchronize(work));
  return leave();
}

int Handle::export_lp(int64_t* row_ptr, int32_t* col_h, double* val_h, double* c_h, double* xl_h, double* xu_h,
                      double* lo_h, double* hi_h) {
  SCUC_TRY(enter());
  cudaStream_t s = work;
  std::vector<int> rp32(m + 1);
  SCUC_CUDA(cudaMemcpyAsync(rp32.data(), rp, (m + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (nnz && col_h) SCUC_CUDA(cudaMemcpyAsync(col_h, col, nnz * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (nnz && val_h) SCUC_CUDA(cudaMemcpyAsync(val_h, val, nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (n && c_h) SCUC_CUDA(cudaMemcpyAsync(c_h, c, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (n && xl_h) SCUC_CUDA(cudaMemcpyAsync(xl_h, xl, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (n && xu_h) SCUC_CUDA(cudaMemcpyAsync(xu_h, xu, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (m && lo_h) SCUC_CUDA(cudaMemcpyAsync(lo_h, lo, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (m && hi_h) SCUC_CUDA(cudaMemcpyAsync(hi_h, hi, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  SCUC_CUDA(cudaStreamSynchronize(s));
  if (row_ptr)
    for (int i = 0; i <= m; i++) row_ptr[i] = rp32[i];
  return leave();
}

}  // namespace scuc

using scuc::Handle;

extern "C" {

void scuc_default_fix_params(scuc_fix_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->tau = 0.1;
  p->t_first = 1;
  p->max_passes = 100;
  p->x_on_device = 0;
  p->build_reduced = 1;
}

int scuc_fix_and_propagate(scuc_lp* lp, const scuc_map* map, const uint8_t* is_int, const double* x_relaxed,
                           const scuc_fix_params* p, int8_t* fix_out, scuc_lp** reduced_out,
                           int32_t* col_map_out, int32_t* row_map_out, scuc_fix_info* info) {
  if (!lp || !lp->h || !map) {
    scuc::set_error("scuc_fix_and_propagate: null argument");
    return SCUC_E_INVALID;
  }
  scuc_fix_params d;
  if (!p) {
    scuc_default_fix_params(&d);
    p = &d;
  }
  if (reduced_out) *reduced_out = nullptr;
  Handle* red = nullptr;
  const int rc = lp->h->fix_and_propagate(*map, is_int, x_relaxed, *p, fix_out,
                                          (reduced_out && p->build_reduced) ? &red : nullptr, col_map_out,
                                          row_map_out, info);
  if (red) *reduced_out = new scuc_lp{red};
  return rc;
}

int scuc_lp_get_bounds(const scuc_lp* lp, double* xl, double* xu) {
  if (!lp || !lp->h) {
    scuc::set_error("null handle");
    return SCUC_E_INVALID;
  }
  return lp->h->get_bounds(xl, xu);
}

int scuc_lp_set_bounds(scuc_lp* lp, const double* xl, const double* xu, int32_t on_device) {
  if (!lp || !lp->h || (lp->h->n > 0 && (!xl || !xu))) {
    scuc::set_error("scuc_lp_set_bounds: null argument");
    return SCUC_E_INVALID;
  }
  return lp->h->set_bounds(xl, xu, on_device);
}

int scuc_lp_export(const scuc_lp* lp, int64_t* row_ptr, int32_t* col, double* val, double* c, double* xl,
                   double* xu, double* lo, double* hi) {
  if (!lp || !lp->h) {
    scuc::set_error("null handle");
    return SCUC_E_INVALID;
  }
  return lp->h->export_lp(row_ptr, col, val, c, xl, xu, lo, hi);
}

}  // extern "C"
