// KKT residuals of a caller-supplied point, computed without allocating any
// device memory (scuc_lp_kkt_noalloc in include/scuc_lp.h).
//
// The two residual SpMVs write one partial sum per row block; those partials
// live in a file-scope device array instead of memory obtained from
// cudaMalloc, so a call allocates nothing.  Every GPU that loads this library
// holds the array (8 MiB) until the process exits.
#include <cmath>
#include <mutex>

#include "lp.h"
#include "spmv.cuh"

namespace scuc {
namespace {

// partial-sum slots: 3 per row block of A plus 4 per row block of A^T
constexpr int kNoallocSlots = 1 << 20;
static __device__ __align__(256) double g_kkt_scratch[kNoallocSlots];

constexpr int kMaxDevices = 256;
std::mutex g_addr_mu;
// device address of g_kkt_scratch, per device, with the ID of the context it
// was looked up in: a device reset ends that context, the next context loads
// the module again (possibly at another address) and has another ID
double* g_addr[kMaxDevices] = {};
unsigned long long g_addr_ctx[kMaxDevices] = {};

typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

// ID of the current context (driver calls reached through the runtime, so the
// library links no driver library); 0 when unavailable
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    looked_up = true;
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array in the current context, looked up once
// per device and context (the device must be current).  In host code the
// array's name is only a host-side stand-in, never a device address.
int scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("device ordinal %d out of range", device);
    return SCUC_E_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_addr_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_addr[device] || ctx == 0 || ctx != g_addr_ctx[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_kkt_scratch);
    if (e != cudaSuccess || !p) {
      set_error("cudaGetSymbolAddress of the residual scratch failed on device %d: %s", device,
                cudaGetErrorString(e));
      return SCUC_E_CUDA;
    }
    g_addr[device] = static_cast<double*>(p);
    g_addr_ctx[device] = ctx;
  }
  *out = g_addr[device];
  return SCUC_OK;
}

__device__ __forceinline__ double clamp_box(double v, double l, double u) {
  return v < l ? l : (v > u ? u : v);
}

__device__ __forceinline__ double finite_mag(double lo, double hi) {
  double b = 0.0;
  if (isfinite(lo) && fabs(lo) > b) b = fabs(lo);
  if (isfinite(hi) && fabs(hi) > b) b = fabs(hi);
  return b;
}

// rows of A: (A x)_i -> violation of [lo_i, hi_i], |b|^2, y-part of the dual objective
struct RowEpi {
  const double *lo, *hi, *y;
  double acc[3];
  __device__ void load(int) {}
  __device__ void row(int i, double a) {
    const double l = lo[i], h = hi[i];
    const double v = a - clamp_box(a, l, h);
    acc[0] += v * v;
    const double b = finite_mag(l, h);
    acc[1] += b * b;
    const double yi = y[i];
    if (yi > 0.0 && isfinite(l)) acc[2] += l * yi;
    else if (yi < 0.0 && isfinite(h)) acc[2] += h * yi;
  }
};

// rows of A^T: (A^T y)_j -> dual residual, |c|^2, primal objective, z-part of the dual objective
struct ColEpi {
  const double *c, *xl, *xu, *x, *z;
  double acc[4];
  __device__ void load(int) {}
  __device__ void row(int j, double g) {
    const double cj = c[j], zj = z[j];
    const double d = cj - g - zj;
    acc[0] += d * d;
    acc[1] += cj * cj;
    acc[2] += cj * x[j];
    if (zj > 0.0 && isfinite(xl[j])) acc[3] += xl[j] * zj;
    else if (zj < 0.0 && isfinite(xu[j])) acc[3] += xu[j] * zj;
  }
};

__global__ void __launch_bounds__(kBlock) k_kkt_rows(const int* __restrict__ rp, const int* __restrict__ col,
                                                     const double* __restrict__ val, Partition part,
                                                     const double* __restrict__ x, const double* __restrict__ lo,
                                                     const double* __restrict__ hi, const double* __restrict__ y,
                                                     double* __restrict__ partial) {
  extern __shared__ __align__(128) unsigned char smem[];
  RowEpi epi{lo, hi, y, {0.0, 0.0, 0.0}};
  spmv_block<double>(rp, col, val, x, part, smem, epi);
  block_store<3>(epi.acc, partial, part);
}

__global__ void __launch_bounds__(kBlock) k_kkt_cols(const int* __restrict__ rpt, const int* __restrict__ colt,
                                                     const double* __restrict__ valt, Partition part,
                                                     const double* __restrict__ y, const double* __restrict__ c,
                                                     const double* __restrict__ xl, const double* __restrict__ xu,
                                                     const double* __restrict__ x, const double* __restrict__ z,
                                                     double* __restrict__ partial) {
  extern __shared__ __align__(128) unsigned char smem[];
  ColEpi epi{c, xl, xu, x, z, {0.0, 0.0, 0.0, 0.0}};
  spmv_block<double>(rpt, colt, valt, y, part, smem, epi);
  block_store<4>(epi.acc, partial, part);
}

constexpr int kFinalThreads = 1024;

__device__ double fixed_order_sum(const double* p, int cnt) {
  __shared__ double s_w[kFinalThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < cnt; i += kFinalThreads) s += p[i];
  s = warp_sum(s);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kFinalThreads / 32; w++) r += s_w[w];
  return r;
}

// out = {r_p, r_d, gap, pobj, dobj, kkt}
__global__ void __launch_bounds__(kFinalThreads) k_kkt_final(const double* __restrict__ partial, int nA, int nT,
                                                             double* __restrict__ out) {
  const double viol2 = fixed_order_sum(partial + 0 * nA, nA);
  const double b2 = fixed_order_sum(partial + 1 * nA, nA);
  const double dy = fixed_order_sum(partial + 2 * nA, nA);
  const double* pc = partial + 3 * nA;
  const double dres2 = fixed_order_sum(pc + 0 * nT, nT);
  const double c2 = fixed_order_sum(pc + 1 * nT, nT);
  const double pobj = fixed_order_sum(pc + 2 * nT, nT);
  const double dz = fixed_order_sum(pc + 3 * nT, nT);
  if (threadIdx.x == 0) {
    const double rp = sqrt(viol2) / (1.0 + sqrt(b2));
    const double rd = sqrt(dres2) / (1.0 + sqrt(c2));
    const double dobj = dy + dz;
    const double gap = fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
    out[0] = rp;
    out[1] = rd;
    out[2] = gap;
    out[3] = pobj;
    out[4] = dobj;
    out[5] = (rp != rp || rd != rd || gap != gap) ? (double)NAN : fmax(rp, fmax(rd, gap));  // NaN carried
  }
}

}  // namespace

int Handle::kkt_noalloc(const double* xd, const double* yd, const double* zd, double* out) {
  const int64_t need = 3 * (int64_t)pA.nblk + 4 * (int64_t)pT.nblk;
  if (need > kNoallocSlots) {
    set_error("scuc_lp_kkt_noalloc: this LP needs %lld partial-sum slots (3 x %d row blocks of A + "
              "4 x %d row blocks of A^T); the fixed scratch holds %d",
              (long long)need, pA.nblk, pT.nblk, kNoallocSlots);
    return SCUC_E_INVALID;
  }
  SCUC_TRY(enter());
  double* scratch = nullptr;
  SCUC_TRY(scratch_address(device, &scratch));
  cudaStream_t s = work;
  // every slot read by the final reduction is written by a block first, so
  // nothing left by an earlier call is read
  double* scratch_t = scratch + 3 * (int64_t)pA.nblk;
  if (pA.nchunk) k_chunk_sums<double><<<pA.nchunkblk, kBlock, 0, s>>>(col, val, xd, pA);
  if (pA.nblk) k_kkt_rows<<<pA.nblk, kBlock, pA.smem, s>>>(rp, col, val, pA, xd, lo, hi, yd, scratch);
  if (pT.nchunk) k_chunk_sums<double><<<pT.nchunkblk, kBlock, 0, s>>>(colt, valt, yd, pT);
  if (pT.nblk) k_kkt_cols<<<pT.nblk, kBlock, pT.smem, s>>>(rpt, colt, valt, pT, yd, c, xl, xu, xd, zd, scratch_t);
  k_kkt_final<<<1, kFinalThreads, 0, s>>>(scratch, pA.nblk, pT.nblk, out);
  SCUC_CUDA(cudaGetLastError());
  return leave();
}

}  // namespace scuc

extern "C" int scuc_lp_kkt_noalloc(scuc_lp* lp, const double* x_dev, const double* y_dev,
                                   const double* z_dev, double* out_dev) {
  if (!lp || !lp->h || !out_dev || (lp->h->n > 0 && (!x_dev || !z_dev)) || (lp->h->m > 0 && !y_dev)) {
    scuc::set_error("scuc_lp_kkt_noalloc: null argument");
    return SCUC_E_INVALID;
  }
  return lp->h->kkt_noalloc(x_dev, y_dev, z_dev, out_dev);
}
