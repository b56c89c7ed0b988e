// Transmission filtering (Fig. 1): the LP is solved without the network
// security rows, the rows of a pool violated by the solution are found on
// the device and appended, and the LP is re-solved from the previous point.
// This file holds the two device steps between solves: the violation check
// of a pool at x (one unscaled FP64 product of the pool plus an ordered
// compaction) and the LP with rows appended (a new handle built from device
// copies).
#include <cmath>
#include <cstring>
#include <vector>

#include "lp.h"
#include "setup_kernels.cuh"

namespace scuc {
namespace {

constexpr int kThreads = 256;

int grid_n(int64_t work) {
  const int64_t g = (work + kThreads - 1) / kThreads;
  return (int)(g < 1 ? 1 : g);
}

// Relative violation of each pool row at x: max of (lo - a x) / (1 + |lo|)
// and (a x - hi) / (1 + |hi|) over the finite bounds, 0 when satisfied;
// flag = violation > tol.  The largest violation goes to *worst (the bits of
// a non-negative double order like the double, so an integer max is exact).
__global__ void k_violations(int m, const double* __restrict__ ax, const double* __restrict__ lo,
                             const double* __restrict__ hi, double tol, int* __restrict__ flag,
                             unsigned long long* __restrict__ worst) {
  __shared__ unsigned long long s_max;
  if (threadIdx.x == 0) s_max = 0ull;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < m) {
    const double a = ax[i], l = lo[i], h = hi[i];
    if (isfinite(l) && l - a > 0.0) v = (l - a) / (1.0 + fabs(l));
    if (isfinite(h) && a - h > 0.0) v = fmax(v, (a - h) / (1.0 + fabs(h)));
    flag[i] = v > tol ? 1 : 0;
  }
  if (v > 0.0) atomicMax(&s_max, (unsigned long long)__double_as_longlong(v));
  __syncthreads();
  if (threadIdx.x == 0 && s_max) atomicMax(worst, s_max);
}

// indices of the flagged rows, in row order (pos = exclusive scan of flag)
__global__ void k_compact_flags(int m, const int* __restrict__ flag, const int* __restrict__ pos,
                                int* __restrict__ rows) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m && flag[i]) rows[pos[i]] = i;
}

// entries of the selected pool rows
__global__ void k_sel_len(int count, const int* __restrict__ sel, const int* __restrict__ rp, int* __restrict__ len) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < count) len[k] = rp[sel[k] + 1] - rp[sel[k]];
}

// Appends the selected pool rows after the base's m0 rows (nnz0 entries):
// warp per selected row copies its entries, row bounds and row pointer.
__global__ void __launch_bounds__(kThreads) k_append_rows(int count, const int* __restrict__ sel,
                                                          const int* __restrict__ off, const int* __restrict__ prp,
                                                          const int* __restrict__ pcol,
                                                          const double* __restrict__ pval,
                                                          const double* __restrict__ plo,
                                                          const double* __restrict__ phi, int m0, int nnz0,
                                                          int* __restrict__ rp, int* __restrict__ col,
                                                          double* __restrict__ val, double* __restrict__ lo,
                                                          double* __restrict__ hi) {
  const int k = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (k >= count) return;
  const int r = sel[k], a = prp[r], b = prp[r + 1], dst = nnz0 + off[k];
  for (int e = a + lane; e < b; e += 32) {
    col[dst + (e - a)] = pcol[e];
    val[dst + (e - a)] = pval[e];
  }
  if (lane == 0) {
    rp[m0 + k + 1] = nnz0 + off[k + 1];
    lo[m0 + k] = plo[r];
    hi[m0 + k] = phi[r];
  }
}

}  // namespace

int Handle::row_violations(const double* x_in, int on_device, double tol, int32_t* rows_out, int32_t cap,
                           int32_t* count_out, double* worst_out) {
  if (!x_in || cap < 0 || (cap > 0 && !rows_out) || !(tol >= 0.0)) {
    set_error("scuc_lp_row_violations: invalid argument");
    return SCUC_E_INVALID;
  }
  SCUC_TRY(enter());
  cudaStream_t s = work;
  const double* xd = x_in;
  if (!on_device) {  // qv (n): power-method scratch, free between solves
    SCUC_CUDA(cudaMemcpyAsync(qv, x_in, n * sizeof(double), cudaMemcpyHostToDevice, s));
    xd = qv;
  }
  int *flag = nullptr, *pos = nullptr, *rows = nullptr;
  unsigned long long* worst = nullptr;
  SCUC_TRY(dev_alloc_bytes((void**)&flag, (m + 1) * sizeof(int)));
  struct Free {  // after the stream's work that uses them
    cudaStream_t s;
    void** p[4];
    ~Free() {
      cudaStreamSynchronize(s);
      for (void** q : p)
        if (*q) dev_free(*q);
    }
  } freer{s, {(void**)&flag, (void**)&pos, (void**)&rows, (void**)&worst}};
  SCUC_TRY(dev_alloc_bytes((void**)&pos, (m + 1) * sizeof(int)));
  SCUC_TRY(dev_alloc_bytes((void**)&rows, (m + 1) * sizeof(int)));
  SCUC_TRY(dev_alloc_bytes((void**)&worst, sizeof(unsigned long long)));
  SCUC_CUDA(cudaMemsetAsync(worst, 0, sizeof(unsigned long long), s));
  // a x into uv (m): unscaled FP64 product with the solver's partition
  if (pA.nchunk) k_chunk_sums<double><<<pA.nchunkblk, kBlock, 0, s>>>(col, val, xd, pA);
  if (pA.nblk) k_spmv_plain<<<pA.nblk, kBlock, pA.smem, s>>>(rp, col, val, xd, pA, uv);
  if (m) k_violations<<<grid_n(m), kThreads, 0, s>>>(m, uv, lo, hi, tol, flag, worst);
  SCUC_CUDA(cudaGetLastError());
  SCUC_TRY(exclusive_scan(flag, m, pos, s));
  if (m) k_compact_flags<<<grid_n(m), kThreads, 0, s>>>(m, flag, pos, rows);
  SCUC_CUDA(cudaGetLastError());
  int cnt = 0;
  unsigned long long wb = 0;
  SCUC_CUDA(cudaMemcpyAsync(&cnt, pos + m, sizeof(int), cudaMemcpyDeviceToHost, s));
  SCUC_CUDA(cudaMemcpyAsync(&wb, worst, sizeof(wb), cudaMemcpyDeviceToHost, s));
  SCUC_CUDA(cudaStreamSynchronize(s));
  const int k = cnt < cap ? cnt : cap;
  if (k > 0) SCUC_CUDA(cudaMemcpy(rows_out, rows, k * sizeof(int), cudaMemcpyDeviceToHost));
  if (count_out) *count_out = cnt;
  if (worst_out) {
    double w;
    memcpy(&w, &wb, sizeof(w));
    *worst_out = w;
  }
  return leave();
}

int Handle::add_rows(const Handle& pool, const int32_t* sel_h, int32_t count, Handle** out) {
  if (pool.n != n || pool.device != device || count < 0 || (count > 0 && !sel_h) || !out) {
    set_error("scuc_lp_add_rows: the pool must have the base's columns and device");
    return SCUC_E_INVALID;
  }
  for (int32_t k = 0; k < count; k++)
    if (sel_h[k] < 0 || sel_h[k] >= pool.m) {
      set_error("scuc_lp_add_rows: row %d of the pool out of range at %d", sel_h[k], k);
      return SCUC_E_INVALID;
    }
  if ((int64_t)m + count > INT32_MAX) {
    set_error("scuc_lp_add_rows: too many rows");
    return SCUC_E_INVALID;
  }
  SCUC_TRY(enter());
  cudaStream_t s = work;
  int *sel = nullptr, *len = nullptr, *off = nullptr;
  SCUC_TRY(dev_alloc_bytes((void**)&sel, (count + 1) * sizeof(int)));
  struct Free {  // after the stream's work that uses them
    cudaStream_t s;
    void** p[3];
    ~Free() {
      cudaStreamSynchronize(s);
      for (void** q : p)
        if (*q) dev_free(*q);
    }
  } freer{s, {(void**)&sel, (void**)&len, (void**)&off}};
  SCUC_TRY(dev_alloc_bytes((void**)&len, (count + 1) * sizeof(int)));
  SCUC_TRY(dev_alloc_bytes((void**)&off, (count + 1) * sizeof(int)));
  if (count) SCUC_CUDA(cudaMemcpyAsync(sel, sel_h, count * sizeof(int), cudaMemcpyHostToDevice, s));
  // the pool's row pointers are read on its own arrays; both handles are on
  // this device and the pool is not being solved (handles are not thread-safe)
  if (count) k_sel_len<<<grid_n(count), kThreads, 0, s>>>(count, sel, pool.rp, len);
  SCUC_CUDA(cudaGetLastError());
  SCUC_TRY(exclusive_scan(len, count, off, s));
  int added = 0;
  SCUC_CUDA(cudaMemcpyAsync(&added, off + count, sizeof(int), cudaMemcpyDeviceToHost, s));
  SCUC_CUDA(cudaStreamSynchronize(s));
  if ((int64_t)nnz + added > INT32_MAX) {
    set_error("scuc_lp_add_rows: too many nonzeros");
    return SCUC_E_INVALID;
  }
  const int m1 = m + count;
  const int64_t nnz1 = nnz + added;
  void *d_rp = nullptr, *d_col = nullptr, *d_val = nullptr, *d_c = nullptr, *d_xl = nullptr, *d_xu = nullptr,
       *d_lo = nullptr, *d_hi = nullptr;
  std::vector<void*> owned;
  struct FreeOwned {  // arrays not passed to a new handle, after the stream's work
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
  SCUC_TRY(oalloc(&d_rp, (m1 + 1) * sizeof(int)));
  SCUC_TRY(oalloc(&d_col, nnz1 * sizeof(int)));
  SCUC_TRY(oalloc(&d_val, nnz1 * sizeof(double)));
  SCUC_TRY(oalloc(&d_c, n * sizeof(double)));
  SCUC_TRY(oalloc(&d_xl, n * sizeof(double)));
  SCUC_TRY(oalloc(&d_xu, n * sizeof(double)));
  SCUC_TRY(oalloc(&d_lo, m1 * sizeof(double)));
  SCUC_TRY(oalloc(&d_hi, m1 * sizeof(double)));
  // the base as it stands (its current column bounds), then the pool rows
  SCUC_CUDA(cudaMemcpyAsync(d_rp, rp, (m + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (nnz) {
    SCUC_CUDA(cudaMemcpyAsync(d_col, col, nnz * sizeof(int), cudaMemcpyDeviceToDevice, s));
    SCUC_CUDA(cudaMemcpyAsync(d_val, val, nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (n) {
    SCUC_CUDA(cudaMemcpyAsync(d_c, c, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SCUC_CUDA(cudaMemcpyAsync(d_xl, xl, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SCUC_CUDA(cudaMemcpyAsync(d_xu, xu, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (m) {
    SCUC_CUDA(cudaMemcpyAsync(d_lo, lo, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SCUC_CUDA(cudaMemcpyAsync(d_hi, hi, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (count)
    k_append_rows<<<grid_n((int64_t)count * 32), kThreads, 0, s>>>(
        count, sel, off, pool.rp, pool.col, pool.val, pool.lo, pool.hi, m, (int)nnz, static_cast<int*>(d_rp),
        static_cast<int*>(d_col), static_cast<double*>(d_val), static_cast<double*>(d_lo),
        static_cast<double*>(d_hi));
  SCUC_CUDA(cudaGetLastError());
  SCUC_CUDA(cudaStreamSynchronize(s));
  owned.clear();  // the new handle frees them, also when its set-up fails
  Handle* H = new Handle();
  const int rc = H->init_device(m1, n, nnz1, static_cast<int*>(d_rp), static_cast<int*>(d_col),
                                static_cast<double*>(d_val), static_cast<double*>(d_c), static_cast<double*>(d_xl),
                                static_cast<double*>(d_xu), static_cast<double*>(d_lo),
                                static_cast<double*>(d_hi), user);
  if (rc != SCUC_OK) {
    delete H;
    return rc;
  }
  *out = H;
  return leave();
}

}  // namespace scuc

using scuc::Handle;

extern "C" {

int scuc_lp_row_violations(scuc_lp* pool, const double* x, int32_t x_on_device, double tol, int32_t* rows_out,
                           int32_t cap, int32_t* count_out, double* worst_out) {
  if (!pool || !pool->h) {
    scuc::set_error("scuc_lp_row_violations: null handle");
    return SCUC_E_INVALID;
  }
  return pool->h->row_violations(x, x_on_device, tol, rows_out, cap, count_out, worst_out);
}

int scuc_lp_add_rows(scuc_lp* base, scuc_lp* pool, const int32_t* rows, int32_t count, scuc_lp** out) {
  if (!base || !base->h || !pool || !pool->h || !out) {
    scuc::set_error("scuc_lp_add_rows: null argument");
    return SCUC_E_INVALID;
  }
  *out = nullptr;
  Handle* H = nullptr;
  const int rc = base->h->add_rows(*pool->h, rows, count, &H);
  if (H) *out = new scuc_lp{H};
  return rc;
}

}  // extern "C"
