// Host side of the SCUC LP library: handle lifetime, device setup, the
// restarted HPR solve loop (Eq. 9) and the C ABI of include/scuc_lp.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <mutex>
#include <string>
#include <thread>
#include <vector>
#include <algorithm>

#include "lp.h"
#include "setup_kernels.cuh"

namespace scuc {

static thread_local std::string g_err;
void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

// Device memory of the library comes from one stream-ordered pool per
// device that keeps freed blocks for reuse (release threshold: never), so
// the handles and temporaries of successive fixing rounds are served from
// memory already mapped, and a free does not synchronise the device as
// cudaFree does.  Allocations and frees are ordered on an internal stream;
// an allocation waits for that stream (usually idle) so the block can be
// used from any stream at once.  A caller frees a block only after the work
// that uses it has completed.
namespace {
constexpr int kMaxPoolDevices = 256;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxPoolDevices] = {};
cudaStream_t g_pool_stream[kMaxPoolDevices] = {};

int pool_for(int dev, cudaMemPool_t* pool, cudaStream_t* st) {
  if (dev < 0 || dev >= kMaxPoolDevices) {
    set_error("device ordinal %d out of range", dev);
    return SCUC_E_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t q = nullptr;
    SCUC_CUDA(cudaMemPoolCreate(&q, &props));
    uint64_t keep = UINT64_MAX;
    SCUC_CUDA(cudaMemPoolSetAttribute(q, cudaMemPoolAttrReleaseThreshold, &keep));
    SCUC_CUDA(cudaStreamCreateWithFlags(&g_pool_stream[dev], cudaStreamNonBlocking));
    g_pool[dev] = q;
  }
  *pool = g_pool[dev];
  *st = g_pool_stream[dev];
  return SCUC_OK;
}
}  // namespace

int dev_alloc_bytes(void** p, size_t bytes) {
  *p = nullptr;
  int dev = 0;
  SCUC_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  cudaStream_t st;
  SCUC_TRY(pool_for(dev, &pool, &st));
  SCUC_CUDA(cudaMallocFromPoolAsync(p, bytes + 64, pool, st));  // padding: aligned bulk copies
  SCUC_CUDA(cudaStreamSynchronize(st));
  return SCUC_OK;
}

void dev_free(void* p) {
  if (!p) return;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return;
  }
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != a.device) cudaSetDevice(a.device);
  cudaMemPool_t pool;
  cudaStream_t st;
  if (pool_for(a.device, &pool, &st) == SCUC_OK) cudaFreeAsync(p, st);
  if (cur >= 0 && cur != a.device) cudaSetDevice(cur);
}

template <typename T>
static int dalloc(T** p, size_t count) {
  void* q = nullptr;
  SCUC_TRY(dev_alloc_bytes(&q, (count ? count : 1) * sizeof(T)));
  *p = static_cast<T*>(q);
  return SCUC_OK;
}

static int grid_for(int64_t work, int block = kBlock) {
  int64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 148 * 16) g = 148 * 16;
  return (int)g;
}

// out[0..n] = exclusive prefix sums of in[0..n-1], out[n] the total
// (recursive over block sums); stream ordered on s, no host synchronisation
int exclusive_scan(const int* in, int n, int* out, cudaStream_t s) {
  const int nb = (n + kScan - 1) / kScan;
  int* scratch = nullptr;  // block sums (nb), their offsets (nb + 1)
  SCUC_CUDA(cudaMallocAsync((void**)&scratch, (2 * (size_t)nb + 2) * sizeof(int), s));
  int *bsum = scratch, *boff = scratch + nb;
  if (n > 0) k_scan_block<<<nb, kScan, 0, s>>>(in, n, out, bsum);
  SCUC_CUDA(cudaGetLastError());
  int rc = SCUC_OK;
  if (nb > 1) {
    rc = exclusive_scan(bsum, nb, boff, s);
    if (rc == SCUC_OK) k_scan_add<<<nb, kScan, 0, s>>>(out, n, boff);
  }
  if (rc == SCUC_OK) k_scan_total<<<1, 32, 0, s>>>(in, n, out);
  cudaFreeAsync(scratch, s);
  SCUC_TRY(rc);
  SCUC_CUDA(cudaGetLastError());
  return SCUC_OK;
}

Handle::~Handle() {
  // the handle's kernels run on work (and graphs launched on it); none may
  // still read its memory when it returns to the pool
  if (work) cudaStreamSynchronize(work);
  for (void* p : allocs) dev_free(p);
  if (graph_exec) cudaGraphExecDestroy(graph_exec);
  for (auto& e : prof_ev) cudaEventDestroy(e);
  if (ctrl_h) cudaFreeHost(ctrl_h);
  if (pctrl_host) cudaFreeHost(pctrl_host);
  if (ev_power) cudaEventDestroy(ev_power);
  if (ev_user) cudaEventDestroy(ev_user);
  if (ev_work) cudaEventDestroy(ev_work);
  for (auto& e : ev_slot)
    if (e) cudaEventDestroy(e);
  if (aux) cudaStreamDestroy(aux);
  if (work) cudaStreamDestroy(work);
}

template <typename T>
int Handle::alloc(T** p, size_t count) {
  SCUC_TRY(dalloc(p, count));
  allocs.push_back((void*)*p);
  return SCUC_OK;
}
// element types other files allocate through a handle
template int Handle::alloc<int>(int**, size_t);
template int Handle::alloc<double>(double**, size_t);
template int Handle::alloc<float>(float**, size_t);

// ---------------------------------------------------------------------------
// validation (host, before any launch)
// ---------------------------------------------------------------------------
// Input rules of scuc_lp_create, checked on the host before any kernel runs.
// Sizes, pointers and the row pointers first (so no entry outside [0, nnz)
// is read), then the entries and bounds in row / column chunks on host
// threads; the error reported is the one of the first failing row (then
// column), as a sequential pass would find it.
namespace {

struct CheckResult {
  int64_t where = -1;  // first failing row / column of the chunk, -1: none
  std::string msg;
};

void check_rows(int32_t i0, int32_t i1, int32_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                const double* lo, const double* hi, CheckResult* r) {
  char buf[160];
  for (int32_t i = i0; i < i1; i++) {
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
      if (col[e] < 0 || col[e] >= n || (e > row_ptr[i] && col[e] <= col[e - 1])) {
        snprintf(buf, sizeof(buf), "column index out of range or not increasing in row %d", i);
        r->where = i;
        r->msg = buf;
        return;
      }
      if (!std::isfinite(val[e])) {
        snprintf(buf, sizeof(buf), "non-finite matrix value in row %d", i);
        r->where = i;
        r->msg = buf;
        return;
      }
    }
    if (std::isnan(lo[i]) || std::isnan(hi[i]) || lo[i] > hi[i] || lo[i] == INFINITY || hi[i] == -INFINITY) {
      snprintf(buf, sizeof(buf), "invalid row bounds at row %d", i);
      r->where = i;
      r->msg = buf;
      return;
    }
  }
}

void check_cols(int32_t j0, int32_t j1, const double* c, const double* xl, const double* xu, CheckResult* r) {
  char buf[160];
  for (int32_t j = j0; j < j1; j++)
    if (!std::isfinite(c[j]) || std::isnan(xl[j]) || std::isnan(xu[j]) || xl[j] > xu[j] || xl[j] == INFINITY ||
        xu[j] == -INFINITY) {
      snprintf(buf, sizeof(buf), "invalid cost or bounds at column %d", j);
      r->where = j;
      r->msg = buf;
      return;
    }
}

}  // namespace

// Entries, row boxes and columns checked by up to 32 host threads (row
// chunks of about equal nonzeros).  Runs while the caller copies the arrays
// to the device; join() returns the first error.
struct Validator {
  std::vector<std::thread> threads;
  std::vector<CheckResult> rows, cols;
  void start(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col, const double* val,
             const double* c, const double* xl, const double* xu, const double* lo, const double* hi) {
    const unsigned hw = std::thread::hardware_concurrency();
    int k = (int)std::min<int64_t>(std::max<unsigned>(hw, 1u), 32);
    if (nnz + m + n < (int64_t)1 << 20) k = 1;
    rows.assign(k, CheckResult{});
    cols.assign(k, CheckResult{});
    int32_t r0 = 0;
    for (int t = 0; t < k; t++) {
      // last row of chunk t: the first row whose start reaches (t+1)/k of the entries
      int32_t r1 = t == k - 1 ? m
                              : (int32_t)(std::lower_bound(row_ptr, row_ptr + m + 1, nnz * (t + 1) / k) - row_ptr);
      r1 = std::max(r0, std::min(r1, m));
      const int32_t c0 = (int32_t)((int64_t)n * t / k), c1 = (int32_t)((int64_t)n * (t + 1) / k);
      threads.emplace_back([=] {
        check_rows(r0, r1, n, row_ptr, col, val, lo, hi, &rows[t]);
        check_cols(c0, c1, c, xl, xu, &cols[t]);
      });
      r0 = r1;
    }
  }
  int join() {
    for (auto& th : threads) th.join();
    threads.clear();
    for (const auto* v : {&rows, &cols})
      for (const CheckResult& r : *v)
        if (r.where >= 0) {
          set_error("%s", r.msg.c_str());
          return SCUC_E_INVALID;
        }
    return SCUC_OK;
  }
  ~Validator() {
    for (auto& th : threads)
      if (th.joinable()) th.join();
  }
};


// sizes, pointers and the row pointers (nondecreasing from 0 to nnz)
static int validate_shape(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                          const double* val, const double* c, const double* xl, const double* xu, const double* lo,
                          const double* hi) {
  if (m < 0 || n < 0 || nnz < 0 || nnz >= (int64_t)INT32_MAX) {
    set_error("invalid sizes m=%d n=%d nnz=%lld", m, n, (long long)nnz);
    return SCUC_E_INVALID;
  }
  if (!row_ptr || (nnz > 0 && (!col || !val)) || (n > 0 && (!c || !xl || !xu)) ||
      (m > 0 && (!lo || !hi))) {
    set_error("null input array");
    return SCUC_E_INVALID;
  }
  if (row_ptr[0] != 0 || row_ptr[m] != nnz) {
    set_error("row_ptr[0] must be 0 and row_ptr[m] must equal nnz");
    return SCUC_E_INVALID;
  }
  for (int32_t i = 0; i < m; i++)
    if (row_ptr[i + 1] < row_ptr[i]) {
      set_error("row_ptr decreases at row %d", i);
      return SCUC_E_INVALID;
    }
  return SCUC_OK;
}

int create_handle(Handle** out, int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                  const int32_t* col, const double* val, const double* c, const double* xl,
                  const double* xu, const double* lo, const double* hi, void* stream) {
  SCUC_TRY(validate_shape(m, n, nnz, row_ptr, col, val, c, xl, xu, lo, hi));
  // the entries are checked while they are copied; no kernel runs before the
  // check has passed
  Validator V;
  V.start(m, n, nnz, row_ptr, col, val, c, xl, xu, lo, hi);
  Handle* H = new Handle();
  int rc = H->init(m, n, nnz, row_ptr, col, val, c, xl, xu, lo, hi, (cudaStream_t)stream, &V);
  if (rc != SCUC_OK) {
    delete H;
    return rc;
  }
  *out = H;
  return SCUC_OK;
}

int Handle::init(int32_t m_, int32_t n_, int64_t nnz_, const int64_t* row_ptr, const int32_t* col_,
                 const double* val_, const double* c_, const double* xl_, const double* xu_,
                 const double* lo_, const double* hi_, cudaStream_t user_, Validator* check) {
  SCUC_TRY(begin(m_, n_, nnz_, user_));
  cudaStream_t s = work;

  std::vector<int> rp32(m + 1);
  for (int i = 0; i <= m; i++) rp32[i] = (int)row_ptr[i];
  SCUC_TRY(alloc(&rp, m + 1));
  SCUC_TRY(alloc(&col, nnz));
  SCUC_TRY(alloc(&val, nnz));
  SCUC_TRY(alloc(&c, n));
  SCUC_TRY(alloc(&xl, n));
  SCUC_TRY(alloc(&xu, n));
  SCUC_TRY(alloc(&lo, m));
  SCUC_TRY(alloc(&hi, m));
  SCUC_CUDA(cudaMemcpyAsync(rp, rp32.data(), (m + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  if (nnz) {
    // Large arrays are page-locked for the copy (register + DMA + unregister
    // measured 64 ms against 122 ms for a pageable copy of the 13k-bus
    // matrix) and released before returning; the next array is registered
    // while the previous one is copied.  If registration fails (memory
    // already registered by the caller, or not registrable) the copy is a
    // plain pageable one.
    const void* srcs[2] = {col_, val_};
    void* dsts[2] = {col, val};
    const size_t sizes[2] = {nnz * sizeof(int), nnz * sizeof(double)};
    bool pinned[2] = {false, false};
    int rc = SCUC_OK;
    for (int k = 0; k < 2 && rc == SCUC_OK; k++) {
      if (sizes[k] >= ((size_t)64 << 20)) {
        if (cudaHostRegister(const_cast<void*>(srcs[k]), sizes[k], cudaHostRegisterDefault) == cudaSuccess)
          pinned[k] = true;
        else
          (void)cudaGetLastError();  // not registrable: pageable copy
      }
      if (cudaMemcpyAsync(dsts[k], srcs[k], sizes[k], cudaMemcpyHostToDevice, s) != cudaSuccess) {
        set_error("host-to-device copy of the matrix failed");
        rc = SCUC_E_CUDA;
      }
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    for (int k = 0; k < 2; k++)
      if (pinned[k]) cudaHostUnregister(const_cast<void*>(srcs[k]));
    SCUC_TRY(rc);
    SCUC_CUDA(e);
  }
  if (n) {
    SCUC_CUDA(cudaMemcpyAsync(c, c_, n * sizeof(double), cudaMemcpyHostToDevice, s));
    SCUC_CUDA(cudaMemcpyAsync(xl, xl_, n * sizeof(double), cudaMemcpyHostToDevice, s));
    SCUC_CUDA(cudaMemcpyAsync(xu, xu_, n * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  if (m) {
    SCUC_CUDA(cudaMemcpyAsync(lo, lo_, m * sizeof(double), cudaMemcpyHostToDevice, s));
    SCUC_CUDA(cudaMemcpyAsync(hi, hi_, m * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  if (check) SCUC_TRY(check->join());
  return setup_device(rp32);
}

int Handle::begin(int32_t m_, int32_t n_, int64_t nnz_, cudaStream_t user_) {
  m = m_;
  n = n_;
  nnz = nnz_;
  user = user_;
  SCUC_CUDA(cudaGetDevice(&device));
  SCUC_CUDA(cudaStreamCreateWithFlags(&work, cudaStreamNonBlocking));
  SCUC_CUDA(cudaEventCreateWithFlags(&ev_user, cudaEventDisableTiming));
  SCUC_CUDA(cudaEventCreateWithFlags(&ev_work, cudaEventDisableTiming));
  SCUC_CUDA(cudaEventCreateWithFlags(&ev_slot[0], cudaEventDisableTiming));
  SCUC_CUDA(cudaEventCreateWithFlags(&ev_slot[1], cudaEventDisableTiming));
  SCUC_CUDA(cudaMallocHost((void**)&ctrl_h, 2 * sizeof(Ctrl)));
  return enter();
}

// Adopts device arrays (allocated by the library; ownership moves to the
// handle) that already satisfy the input rules, then builds the device state.
// With t, the transpose (columns sorted by row, permt the CSR position of
// each entry) and both row-pointer arrays are adopted as well.
int Handle::init_device(int32_t m_, int32_t n_, int64_t nnz_, int* d_rp, int* d_col, double* d_val,
                        double* d_c, double* d_xl, double* d_xu, double* d_lo, double* d_hi,
                        cudaStream_t user_, const DevTranspose* t) {
  rp = d_rp; col = d_col; val = d_val; c = d_c; xl = d_xl; xu = d_xu; lo = d_lo; hi = d_hi;
  for (void* p : {(void*)d_rp, (void*)d_col, (void*)d_val, (void*)d_c, (void*)d_xl, (void*)d_xu,
                  (void*)d_lo, (void*)d_hi})
    allocs.push_back(p);
  if (t) {
    rpt = t->rpt; colt = t->colt; permt = t->permt; valt = t->valt;
    for (void* p : {(void*)rpt, (void*)colt, (void*)permt, (void*)valt}) allocs.push_back(p);
  }
  SCUC_TRY(begin(m_, n_, nnz_, user_));
  if (t) return setup_solver(*t->rp_h, *t->rpt_h);
  std::vector<int> rp32(m + 1);
  SCUC_CUDA(cudaMemcpyAsync(rp32.data(), rp, (m + 1) * sizeof(int), cudaMemcpyDeviceToHost, work));
  SCUC_CUDA(cudaStreamSynchronize(work));
  return setup_device(rp32);
}

// transpose, partitions and solver buffers (data already on the device);
// rp32 is moved from
int Handle::setup_device(std::vector<int>& rp32) {
  std::vector<int> rpt_h;
  SCUC_TRY(build_transpose(&rpt_h));
  return setup_solver(rp32, rpt_h);
}

// A^T in CSR form: count, scan, scatter, per-column sort by row, gather values
int Handle::build_transpose(std::vector<int>* rpt_out) {
  cudaStream_t s = work;

  // transpose: count, scan, scatter, per-column sort by row, gather values
  SCUC_TRY(alloc(&rpt, n + 1));
  SCUC_TRY(alloc(&colt, nnz));
  SCUC_TRY(alloc(&permt, nnz));
  SCUC_TRY(alloc(&valt, nnz));
  int* cnt = nullptr;
  SCUC_TRY(alloc(&cnt, n + 1));
  SCUC_CUDA(cudaMemsetAsync(cnt, 0, (n + 1) * sizeof(int), s));
  if (nnz) k_count_cols<<<grid_for(nnz), kBlock, 0, s>>>(col, nnz, cnt);
  SCUC_CUDA(cudaGetLastError());
  SCUC_TRY(exclusive_scan(cnt, n, rpt, s));
  SCUC_CUDA(cudaMemcpyAsync(cnt, rpt, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (m) k_scatter_t<<<grid_for((int64_t)m * 32), kBlock, 0, s>>>(rp, col, m, cnt, colt, permt);
  SCUC_CUDA(cudaGetLastError());
  std::vector<int> rpt_h(n + 1);
  SCUC_CUDA(cudaMemcpyAsync(rpt_h.data(), rpt, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  SCUC_CUDA(cudaStreamSynchronize(s));
  std::vector<int> longcols;
  for (int j = 0; j < n; j++) {
    const int L = rpt_h[j + 1] - rpt_h[j];
    if (L > kSortCap) {
      set_error("column %d has %d nonzeros; at most %d per column are supported", j, L, kSortCap);
      return SCUC_E_INVALID;
    }
    if (L > 32) longcols.push_back(j);
  }
  if (n) k_sort_small<<<(n + kBlock - 1) / kBlock, kBlock, 0, s>>>(rpt, n, colt, permt);
  SCUC_CUDA(cudaGetLastError());
  if (!longcols.empty()) {
    int* lc = nullptr;
    SCUC_TRY(alloc(&lc, longcols.size()));
    SCUC_CUDA(cudaMemcpyAsync(lc, longcols.data(), longcols.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    SCUC_CUDA(cudaFuncSetAttribute(k_sort_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kSortCap * 8));
    k_sort_block<<<(int)longcols.size(), 1024, kSortCap * 8, s>>>(rpt, lc, colt, permt);
    SCUC_CUDA(cudaGetLastError());
  }
  if (nnz) k_gather_t<<<grid_for(nnz), kBlock, 0, s>>>(permt, nnz, val, valt);
  SCUC_CUDA(cudaGetLastError());
  *rpt_out = std::move(rpt_h);
  return SCUC_OK;
}

// partitions and solver buffers; rp32 / rpt_h: row pointers of A and A^T,
// moved from (kept for the sliced copies of the first solve)
int Handle::setup_solver(std::vector<int>& rp32, std::vector<int>& rpt_h) {
  cudaStream_t s = work;
  // rows above kSellMaxLen are chunked (warp per 512 entries); the sliced
  // ELL copies below hold the rest for the iteration products
  SCUC_TRY(build_partition(rp32, m, &pA, kSellMaxLen));
  SCUC_TRY(build_partition(rpt_h, n, &pT, kSellMaxLen));
  // the sliced ELL copy of A^T (primal step) is built at the first solve
  // that uses it (a reduced LP that is only exported or batched never
  // needs it); the row pointers are kept until then.  The dual step stays
  // on the CSR partition: its short rows are staged runs, its long rows
  // chunks (measured faster than a sliced copy of A's short rows plus an
  // elementwise update on the 13k-bus LP: 0.199 vs 0.210 ms).
  rpt_plan = std::move(rpt_h);
  if (pA.nchunk) rp_plan = std::move(rp32);
  for (Partition* P : {&pA, &pT})
    for (void* q : {(void*)P->listx, (void*)P->desc, (void*)P->chunks, (void*)P->long_rows, (void*)P->chunk_ptr,
                    (void*)P->cpart, (void*)P->slot})
      if (q) allocs.push_back(q);

  // scaled data and iterates
  SCUC_TRY(alloc(&vs, nnz));
  SCUC_TRY(alloc(&vst, nnz));
  SCUC_TRY(alloc(&Dr, m));
  SCUC_TRY(alloc(&Dc, n));
  SCUC_TRY(alloc(&cs, n));
  SCUC_TRY(alloc(&xls, n));
  SCUC_TRY(alloc(&xus, n));
  SCUC_TRY(alloc(&los, m));
  SCUC_TRY(alloc(&his, m));
  SCUC_TRY(alloc(&x, n));
  SCUC_TRY(alloc(&x0, n));
  SCUC_TRY(alloc(&xt, n));
  SCUC_TRY(alloc(&xbar, n));
  SCUC_TRY(alloc(&zbar, n));
  SCUC_TRY(alloc(&y, m));
  SCUC_TRY(alloc(&y0, m));
  SCUC_TRY(alloc(&ybar, m));
  SCUC_TRY(alloc(&xt32, n));
  SCUC_TRY(alloc(&y32, m));
  epi_gx = (int)std::max<int64_t>(1, std::min<int64_t>(148 * 8, ((int64_t)n + kBlock - 1) / kBlock));
  SCUC_TRY(alloc(&gsum, n));
  SCUC_TRY(alloc(&gsum32, n));
  SCUC_TRY(alloc(&partP, 4 * (size_t)epi_gx));
  SCUC_TRY(alloc(&partD, 2 * (size_t)pA.nblk));
  SCUC_TRY(alloc(&partRA, 6 * (size_t)std::max(pA.nblk, kNormBlocks)));
  SCUC_TRY(alloc(&dychk, m));
  SCUC_TRY(alloc(&dxchk, n));
  SCUC_TRY(alloc(&partRT, 6 * (size_t)std::max(pT.nblk, kNormBlocks)));
  SCUC_TRY(alloc(&ctrl, 1));
  SCUC_TRY(alloc(&pctrl, 1));
  SCUC_TRY(alloc(&qv, n));
  SCUC_TRY(alloc(&uv, m));
  SCUC_TRY(alloc(&wv, n));
  SCUC_CUDA(cudaMemsetAsync(xbar, 0, n * sizeof(double) + 16, s));
  SCUC_CUDA(cudaMemsetAsync(zbar, 0, n * sizeof(double) + 16, s));
  SCUC_CUDA(cudaMemsetAsync(ybar, 0, m * sizeof(double) + 16, s));
  SCUC_CUDA(cudaStreamSynchronize(s));
  return leave();
}

// the handle's private stream follows the caller's stream and vice versa
int Handle::enter() {
  SCUC_CUDA(cudaSetDevice(device));
  SCUC_CUDA(cudaEventRecord(ev_user, user));
  SCUC_CUDA(cudaStreamWaitEvent(work, ev_user, 0));
  return SCUC_OK;
}

int Handle::leave() {
  SCUC_CUDA(cudaEventRecord(ev_work, work));
  SCUC_CUDA(cudaStreamWaitEvent(user, ev_work, 0));
  return SCUC_OK;
}

DevLP Handle::dev() const {
  DevLP L;
  L.m = m; L.n = n;
  L.rp = rp; L.col = col; L.rpt = rpt; L.colt = colt;
  L.vs = vs; L.vst = vst; L.vs32 = vs32; L.vst32 = vst32; L.val = val; L.valt = valt;
  L.c = cs; L.xl = xls; L.xu = xus; L.lo = los; L.hi = his; L.Dr = Dr; L.Dc = Dc;
  L.x = x; L.x0 = x0; L.xt = xt; L.xbar = xbar; L.zbar = zbar; L.y = y; L.y0 = y0; L.ybar = ybar;
  L.xt32 = xt32; L.y32 = y32;
  L.sT = sT;
  L.sA = sA;
  L.qchk = uv; L.dychk = dychk;  // uv: power-method scratch, free during iterations
  L.dxchk = dxchk;
  L.coef = coef; L.coef_w = coef;
  L.partP = partP; L.partD = partD; L.partRA = partRA; L.partRT = partRT;
  L.gsum = gsum;
  L.gsum32 = gsum32;
  L.epi_gx = epi_gx;
  L.pA = pA; L.pT = pT;
  L.ctrl = ctrl; L.log = log_d;
  L.nlp = 1;
  L.blkA = L.blkT = L.ablk0 = L.tblk0 = L.row0 = L.col0 = nullptr;
  L.coef_stride = 0;
  L.log_stride = 0;
  return L;
}

// Pock-Chambolle scaling + normalisation (Sec. 3.A), then the unscaled norms
int Handle::setup_scaling(int use_scaling, bool need_f32) {
  cudaStream_t s = work;
  // D_r = D_c = 1; Ruiz passes (use_scaling = 2); Pock-Chambolle (>= 1).
  // Factors of a pass are computed from the same D, then applied.
  k_fill<<<grid_for(std::max(m, n)), kBlock, 0, s>>>(Dr, m, Dc, n, 1.0);
  const int mb = (m + kBlock - 1) / kBlock, nb = (n + kBlock - 1) / kBlock;
  const int npass = use_scaling == 2 ? 11 : (use_scaling == 1 ? 1 : 0);
  for (int pass = 0; pass < npass; pass++) {
    const int use_max = pass < npass - 1 ? 1 : 0;  // Ruiz passes, then the sum pass
    if (use_max) {
      if (m) k_scale_factor<<<mb, kBlock, 0, s>>>(rp, col, val, m, Dr, Dc, 0, use_max, uv);
      if (n) k_scale_factor<<<nb, kBlock, 0, s>>>(rpt, colt, valt, n, Dr, Dc, 1, use_max, wv);
      nlaunch += (m ? 1 : 0) + (n ? 1 : 0);
    } else {
      // sum pass as two products on the solver's balanced partitions (long
      // rows in chunks): |A| Dc into uv, |A^T| Dr into wv; vs and vst hold
      // |A| and |A^T| until the scaled values overwrite them below
      if (nnz) k_abs2<<<grid_for(nnz), kBlock, 0, s>>>(val, vs, nnz, valt, vst, nnz);
      if (pA.nchunk) k_chunk_sums<double><<<pA.nchunkblk, kBlock, 0, s>>>(col, vs, Dc, pA);
      if (pA.nblk) k_spmv_plain<<<pA.nblk, kBlock, pA.smem, s>>>(rp, col, vs, Dc, pA, uv);
      if (pT.nchunk) k_chunk_sums<double><<<pT.nchunkblk, kBlock, 0, s>>>(colt, vst, Dr, pT);
      if (pT.nblk) k_spmv_plain<<<pT.nblk, kBlock, pT.smem, s>>>(rpt, colt, vst, Dr, pT, wv);
      if (m) k_factor_from_sums<<<mb, kBlock, 0, s>>>(m, Dr, uv, uv);
      if (n) k_factor_from_sums<<<nb, kBlock, 0, s>>>(n, Dc, wv, wv);
      nlaunch += (nnz ? 1 : 0) + (pA.nchunk ? 1 : 0) + (pA.nblk ? 1 : 0) + (pT.nchunk ? 1 : 0) +
                 (pT.nblk ? 1 : 0) + (m ? 1 : 0) + (n ? 1 : 0);
    }
    k_mul2<<<grid_for(std::max(m, n)), kBlock, 0, s>>>(Dr, uv, m, Dc, wv, n);
    nlaunch += 1;
  }
  nlaunch += 1 + (m ? 1 : 0) + (nnz ? 1 : 0) + 4;
  if (m) k_scale_vals<<<grid_for((int64_t)m * 32), kBlock, 0, s>>>(rp, col, val, m, Dr, Dc, vs);
  if (nnz) k_gather_t<<<grid_for(nnz), kBlock, 0, s>>>(permt, nnz, vs, vst);
  k_scale_vecs<<<grid_for(std::max(m, n)), kBlock, 0, s>>>(m, n, Dr, Dc, c, xl, xu, lo, hi, cs, xls, xus,
                                                          los, his);
  k_norms_partial<<<kNormBlocks, kBlock, 0, s>>>(m, n, los, his, cs, lo, hi, c, partRT);
  k_norms_final<<<1, kDecideThreads, 0, s>>>(partRT, kNormBlocks, use_scaling, ctrl);
  k_normalize<<<grid_for(std::max(m, n)), kBlock, 0, s>>>(m, n, ctrl, cs, xls, xus, los, his);
  SCUC_CUDA(cudaGetLastError());
  if (need_f32) {
    if (!vs32) {
      SCUC_TRY(alloc(&vs32, nnz));
      SCUC_TRY(alloc(&vst32, nnz));
      // the FP32 chunk products read a chunk stream of values and 16-bit
      // column offsets (its column part once per handle)
      SCUC_TRY(chunk_stream(&pA, col, 0));
      SCUC_TRY(chunk_stream(&pT, colt, 1));
    }
    if (nnz) {
      k_to_f32<<<grid_for(nnz), kBlock, 0, s>>>(vs, nnz, vs32);
      k_to_f32<<<grid_for(nnz), kBlock, 0, s>>>(vst, nnz, vst32);
      nlaunch += 2;
    }
    if (pA.cst) k_chunk_vals<<<pA.nchunkblk, kBlock, 0, s>>>(vs32, pA);
    if (pT.cst) k_chunk_vals<<<pT.nchunkblk, kBlock, 0, s>>>(vst32, pT);
    nlaunch += (pA.cst ? 1 : 0) + (pT.cst ? 1 : 0);
    SCUC_CUDA(cudaGetLastError());
  }
  if (sT.nslice) {
    k_sell_fill<<<(sT.nslice + kBlock / 32 - 1) / (kBlock / 32), kBlock, 0, s>>>(sT, rpt, colt, vst,
                                                                              need_f32 ? vst32 : nullptr);
    nlaunch += 1;
    SCUC_CUDA(cudaGetLastError());
  }
  if (sA.nslice) {
    k_sell_fill<<<(sA.nslice + kBlock / 32 - 1) / (kBlock / 32), kBlock, 0, s>>>(sA, rp, col, vs,
                                                                              need_f32 ? vs32 : nullptr);
    nlaunch += 1;
    SCUC_CUDA(cudaGetLastError());
  }

  return SCUC_OK;
}

int Handle::chunk_stream(Partition* P, const int* col_d, int which) {
  cudaStream_t s = work;
  if (!P->nchunk || P->cst || !index16) return SCUC_OK;
  if (!n16_d) {
    void* q = nullptr;
    SCUC_TRY(dev_alloc_bytes(&q, 2 * sizeof(unsigned long long)));
    allocs.push_back(q);
    n16_d = static_cast<unsigned long long*>(q);
    SCUC_CUDA(cudaMemsetAsync(n16_d, 0, 2 * sizeof(unsigned long long), s));
  }
  void* q = nullptr;
  SCUC_TRY(dev_alloc_bytes(&q, (size_t)P->nchunk * kChunkRec16 * 16));
  P->cst = static_cast<uint4*>(q);  // freed with the partition
  k_chunk_rec<<<P->nchunkblk, kBlock, 0, s>>>(col_d, *P, n16_d + which);
  nlaunch += 1;
  SCUC_CUDA(cudaGetLastError());
  // pageable destination: returns once the count has arrived (once per handle)
  SCUC_CUDA(cudaMemcpyAsync(&n16_h[which], n16_d + which, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  SCUC_CUDA(cudaStreamSynchronize(s));
  return SCUC_OK;
}

int Handle::sell_values(Sell* S, const int* rp_d, const int* col_d, bool compress) {
  cudaStream_t s = work;
  if (!S->nslice) return SCUC_OK;
  if (compress && index16) {
    int* rec = nullptr;
    int* bad = nullptr;
    SCUC_TRY(alloc(&rec, (size_t)S->nslice * 32 * 4));
    SCUC_TRY(alloc(&bad, 1));
    S->lrec = reinterpret_cast<int4*>(rec);
    SCUC_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    k_sell_lrec<<<(S->nslice + kBlock / 32 - 1) / (kBlock / 32), kBlock, 0, s>>>(*S, rp_d, col_d, bad);
    nlaunch += 1;
    SCUC_CUDA(cudaGetLastError());
    int bad_h = 0;
    SCUC_CUDA(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaStreamSynchronize(s));
    if (!bad_h) {
      float* v = nullptr;
      int* o = nullptr;
      SCUC_TRY(alloc(&v, (size_t)S->npair * 64));
      SCUC_TRY(alloc(&o, (size_t)S->npair * 32));
      S->v2 = reinterpret_cast<float2*>(v);
      S->o2 = reinterpret_cast<unsigned*>(o);
      S->compressed = 1;
      return SCUC_OK;
    }
  }
  int* cv = nullptr;
  SCUC_TRY(alloc(&cv, (size_t)S->nent * 2));
  S->cv32 = reinterpret_cast<int2*>(cv);
  return SCUC_OK;
}

// power method on A_hat (Sec. 3): lambda estimate of lambda_max(A A^T).
// power_start seeds it, power_round queues 16 iterations and a copy of the
// state to pinned host memory, power_poll waits for that copy: a batch runs
// the rounds of all its LPs on their own streams before polling any.
int Handle::power_start(const scuc_solve_params& p) {
  cudaStream_t s = work;
  if (!pctrl_host) SCUC_CUDA(cudaMallocHost((void**)&pctrl_host, sizeof(PowerCtrl)));
  if (!ev_power) SCUC_CUDA(cudaEventCreateWithFlags(&ev_power, cudaEventDisableTiming));
  PowerCtrl P0{};
  P0.tol = p.power_tol;
  P0.max_iter = p.power_max_iter;
  *pctrl_host = P0;
  SCUC_CUDA(cudaMemcpyAsync(pctrl, pctrl_host, sizeof(PowerCtrl), cudaMemcpyHostToDevice, s));
  k_power_seed<<<kNormBlocks, kBlock, 0, s>>>(n, p.power_seed, qv, partRT);
  k_power_seed_norm<<<1, kDecideThreads, 0, s>>>(partRT, kNormBlocks, pctrl);
  // MIXED solves run the products in FP32 (values vs32 / vst32; q in xt32,
  // u = A q in y32: both unused until the iterations start)
  power_f32 = p.precision == SCUC_MIXED && vs32 && vst32;
  // FP32 A^T products on the sliced copy of A^T when the solve uses it
  power_sell = power_f32 && sT.nslice > 0 && p.spmv_layout == 0;
  k_power_norm_seed<<<grid_for(n), kBlock, 0, s>>>(n, qv, power_f32 ? xt32 : nullptr, pctrl);
  nlaunch += 3;
  SCUC_CUDA(cudaGetLastError());
  power_rounds = 0;
  return SCUC_OK;
}

int Handle::power_round(const scuc_solve_params& p) {
  cudaStream_t s = work;
  const bool f32 = power_f32;
  float* q32 = f32 ? xt32 : nullptr;
  for (int j = 0; j < 16; j++) {
    if (f32) {
      if (pA.nchunk) k_power_chunks<float><<<pA.nchunkblk, kBlock, 0, s>>>(col, vs32, q32, pA, pctrl);
      if (pA.nblk)
        k_power_spmv32<<<pA.nblk, kBlock, pA.smem, s>>>(rp, col, vs32, q32, pA, nullptr, y32, partRA, pctrl);
      if (pT.nchunk) k_power_chunks<float><<<pT.nchunkblk, kBlock, 0, s>>>(colt, vst32, y32, pT, pctrl);
      if (pT.nblk && power_sell)
        k_power_sell32<<<std::min(pT.nblk, sell_blocks(sT, pT)), kBlock, 0, s>>>(sT, pT, y32, wv, xt32, partRT,
                                                                                 pctrl);
      else if (pT.nblk)
        k_power_spmv32<<<pT.nblk, kBlock, pT.smem, s>>>(rpt, colt, vst32, y32, pT, wv, xt32, partRT, pctrl);
    } else {
      if (pA.nchunk) k_power_chunks<double><<<pA.nchunkblk, kBlock, 0, s>>>(col, vs, qv, pA, pctrl);
      if (pA.nblk) k_power_spmv<<<pA.nblk, kBlock, pA.smem, s>>>(rp, col, vs, qv, pA, uv, partRA, pctrl);
      if (pT.nchunk) k_power_chunks<double><<<pT.nchunkblk, kBlock, 0, s>>>(colt, vst, uv, pT, pctrl);
      if (pT.nblk) k_power_spmv<<<pT.nblk, kBlock, pT.smem, s>>>(rpt, colt, vst, uv, pT, wv, partRT, pctrl);
    }
    k_power_decide<<<1, kDecideThreads, 0, s>>>(partRA, pA.nblk, partRT, pT.nblk, pctrl);
    k_power_norm<<<grid_for(n), kBlock, 0, s>>>(n, wv, qv, q32, pctrl);
    nlaunch += 2 + (pA.nblk ? 1 : 0) + (pT.nblk ? 1 : 0) + (pA.nchunk ? 1 : 0) + (pT.nchunk ? 1 : 0);
  }
  SCUC_CUDA(cudaGetLastError());
  SCUC_CUDA(cudaMemcpyAsync(pctrl_host, pctrl, sizeof(PowerCtrl), cudaMemcpyDeviceToHost, s));
  SCUC_CUDA(cudaEventRecord(ev_power, s));
  power_rounds++;
  (void)p;
  return SCUC_OK;
}

// after the last queued round: *done once the estimate has converged or
// max_iter iterations have run (the device stops counting there)
int Handle::power_poll(const scuc_solve_params& p, bool* done, double* lam, int* iters) {
  SCUC_CUDA(cudaEventSynchronize(ev_power));
  *done = pctrl_host->done != 0 || power_rounds * 16 >= p.power_max_iter;
  *lam = pctrl_host->lam;
  *iters = pctrl_host->it;
  return SCUC_OK;
}

int Handle::power_method(const scuc_solve_params& p, double* lam_out, int* iters_out) {
  SCUC_TRY(power_start(p));
  bool done = false;
  while (!done) {
    SCUC_TRY(power_round(p));
    SCUC_TRY(power_poll(p, &done, lam_out, iters_out));
  }
  return SCUC_OK;
}

int Handle::ensure_log(int cap) {
  if (cap > log_cap) {
    scuc_check_log* nl = nullptr;
    SCUC_TRY(alloc(&nl, cap));
    log_d = nl;
    log_cap = cap;
  }
  return SCUC_OK;
}

// One check period: anchor, check_every-1 plain iterations, a check iteration,
// the two FP64 residual SpMVs and the decide kernel.
// The check_every iterations of one period in one precision (PREC) on stream
// s; with profile, events around the two half-steps of every iteration.
template <int PREC>
int Handle::launch_iterations(cudaStream_t s, int check_every, bool profile) {
  const DevLP L = dev();
  for (int j = 0; j < check_every; j++) {
    const bool chk = (j == check_every - 1);
    if (profile) SCUC_CUDA(cudaEventRecord(prof_ev[4 * j + 0], s));
    // plain iterations: the update fused into the product's launch
    const bool fuse_p = !chk && !split_steps && use_sell;
    const bool fuse_d = !chk && !split_steps && use_sell_dual;
    if (pT.nchunk) k_chunks_iter<kChunksPrimal, PREC><<<pT.nchunkblk, kBlock, 0, s>>>(L);
    if (use_sell) {
      const int g = (sT.nslice + kPrimalWpb - 1) / kPrimalWpb + (pT.nlong + kPrimalBlock - 1) / kPrimalBlock;
      if (g && fuse_p) k_primal_sell<PREC, true><<<g, kPrimalBlock, 0, s>>>(L, j);
      else if (g) k_primal_sell<PREC, false><<<g, kPrimalBlock, 0, s>>>(L, j);
    } else if (pT.nblk) {
      k_primal_sum<PREC><<<pT.nblk, kBlock, pT.smem, s>>>(L);
    }
    if (chk) k_primal_epi<true, PREC><<<epi_gx, kBlock, 0, s>>>(L, j);
    else if (!fuse_p) k_primal_epi<false, PREC><<<epi_gx, kBlock, 0, s>>>(L, j);
    if (profile) SCUC_CUDA(cudaEventRecord(prof_ev[4 * j + 1], s));
    if (profile) SCUC_CUDA(cudaEventRecord(prof_ev[4 * j + 2], s));
    if (fuse_d) {
      k_dual_fused<PREC><<<(sA.nslice + kDualWpb - 1) / kDualWpb + (pA.nchunk + kDualWpb - 1) / kDualWpb,
                           kDualBlock, 0, s>>>(L, j);
      k_dual_long<PREC><<<(pA.nlong + 63) / 64, 64, 0, s>>>(L, j);
    } else {
      if (pA.nchunk) k_chunks_iter<kChunksDual, PREC><<<pA.nchunkblk, kBlock, 0, s>>>(L);
      if (pA.nblk) {
        if (chk) k_dual<true, PREC><<<pA.nblk, kBlock, pA.smem, s>>>(L, j);
        else k_dual<false, PREC><<<pA.nblk, kBlock, pA.smem, s>>>(L, j);
      }
    }
    if (profile) SCUC_CUDA(cudaEventRecord(prof_ev[4 * j + 3], s));
  }
  SCUC_CUDA(cudaGetLastError());
  return SCUC_OK;
}

// kernels of one period: anchor, iterations, residual SpMVs, decide
int64_t Handle::period_kernels(int check_every) const {
  const int la = (pA.nblk ? 1 : 0) + (pA.nchunk ? 1 : 0), lt = (pT.nblk ? 1 : 0) + (pT.nchunk ? 1 : 0);
  const bool gt = sT.nslice > 0 || pT.nlong > 0;  // k_primal_sell has blocks
  const int lt_iter = use_sell ? (pT.nchunk ? 1 : 0) + (gt ? 1 : 0) : lt;
  // a plain iteration: primal product (+ update unless fused), dual step
  const int plain_p = lt_iter + (!split_steps && use_sell ? 0 : 1);
  const int plain_d = la;  // the fused dual step is two launches as well
  return 2 + (int64_t)(check_every - 1) * (plain_p + plain_d) + (la + lt_iter + 1) + (la + lt) * (detect ? 2 : 1);
}

// check SpMVs (FP64) and the decide kernel of a period
int Handle::launch_checks(cudaStream_t s, int check_every) {
  const DevLP L = dev();
  if (pA.nchunk) k_chunks_iter<kChunksResPrimal, kPrecF64><<<pA.nchunkblk, kBlock, 0, s>>>(L);
  if (pA.nblk) k_res_primal<<<pA.nblk, kBlock, pA.smem, s>>>(L);
  if (pT.nchunk) k_chunks_iter<kChunksResDual, kPrecF64><<<pT.nchunkblk, kBlock, 0, s>>>(L);
  if (pT.nblk) {
    // on the sliced copy of A^T when the solve's primal products use it
    // (the same partial-sum slots as the CSR form)
    const int gs = std::min(pT.nblk, sell_blocks(sT, pT));
    if (use_sell && algo == SCUC_ALGO_PDHG_AVG) k_res_dual_sell<true><<<gs, kBlock, 0, s>>>(L);
    else if (use_sell) k_res_dual_sell<false><<<gs, kBlock, 0, s>>>(L);
    else if (algo == SCUC_ALGO_PDHG_AVG) k_res_dual<true><<<pT.nblk, kBlock, pT.smem, s>>>(L);
    else k_res_dual<false><<<pT.nblk, kBlock, pT.smem, s>>>(L);
  }
  if (detect) {  // certificate products A (x_bar - x), A^T (y_bar - y)
    if (pA.nchunk) k_chunks_iter<kChunksInfRows, kPrecF64><<<pA.nchunkblk, kBlock, 0, s>>>(L);
    if (pA.nblk) k_inf_rows<<<pA.nblk, kBlock, pA.smem, s>>>(L);
    if (pT.nchunk) k_chunks_iter<kChunksInfCols, kPrecF64><<<pT.nchunkblk, kBlock, 0, s>>>(L);
    if (pT.nblk) k_inf_cols<<<pT.nblk, kBlock, pT.smem, s>>>(L);
  }
  k_decide<<<1, kDecideThreads, 0, s>>>(L, check_every);
  SCUC_CUDA(cudaGetLastError());
  return SCUC_OK;
}

// One period launched from the host in the phase the host last saw.
int Handle::launch_period(int check_every, bool profile, bool fp64) {
  cudaStream_t s = work;
  k_anchor<<<grid_for(std::max(m, n)), kBlock, 0, s>>>(dev());
  if (fp64) SCUC_TRY(launch_iterations<kPrecF64>(s, check_every, profile));
  else SCUC_TRY(launch_iterations<kPrecF32>(s, check_every, profile));
  SCUC_TRY(launch_checks(s, check_every));
  nlaunch += period_kernels(check_every);
  return SCUC_OK;
}

// The whole iteration as one graph: WHILE (not stopped) { anchor; IF (FP64
// phase) FP64 iterations ELSE FP32 iterations; checks; decide; conditions }.
// The decide kernel's state picks the branch and ends the loop on the
// device, so a solve is one graph launch with no host round trip.
int Handle::build_solve_graph(int check_every, int phase64) {
  if (!aux) SCUC_CUDA(cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  SCUC_CUDA(cudaGraphCreate(&g, 0));
  struct GraphGuard {
    cudaGraph_t g;
    ~GraphGuard() { if (g) cudaGraphDestroy(g); }
  } guard{g};
  cudaGraphConditionalHandle hloop, hphase;
  SCUC_CUDA(cudaGraphConditionalHandleCreate(&hloop, g, 1, cudaGraphCondAssignDefault));
  SCUC_CUDA(cudaGraphConditionalHandleCreate(&hphase, g, phase64 ? 1 : 0, cudaGraphCondAssignDefault));
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hloop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  SCUC_CUDA(cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  const DevLP L = dev();
  cudaStream_t s = work;
  SCUC_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  k_anchor<<<grid_for(std::max(m, n)), kBlock, 0, s>>>(L);
  // the precision branch, inserted into the capture
  cudaStreamCaptureStatus cst;
  cudaGraph_t capg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cst, nullptr, &capg, &deps, nullptr, &ndeps);
  cudaGraphNodeParams ip = {};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hphase;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 2;
  cudaGraphNode_t inode = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&inode, capg, deps, nullptr, ndeps, &ip);
  if (e == cudaSuccess)
    e = cudaStreamUpdateCaptureDependencies(s, &inode, nullptr, 1, cudaStreamSetCaptureDependencies);
  int rc = e == cudaSuccess ? launch_checks(s, check_every) : SCUC_OK;
  if (e == cudaSuccess && rc == SCUC_OK) k_loop_cond<<<1, kDecideThreads, 0, s>>>(L, hloop, hphase, 1);
  cudaGraph_t cap_out = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(s, &cap_out);
  SCUC_CUDA(e);
  SCUC_TRY(rc);
  SCUC_CUDA(e2);
  // the two branches: [0] FP64 phase, [1] FP32 phase
  for (int br = 0; br < 2; br++) {
    SCUC_CUDA(cudaStreamBeginCaptureToGraph(aux, ip.conditional.phGraph_out[br], nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
    rc = br == 0 ? launch_iterations<kPrecF64>(aux, check_every, false)
                 : launch_iterations<kPrecF32>(aux, check_every, false);
    cudaGraph_t bout = nullptr;
    const cudaError_t e3 = cudaStreamEndCapture(aux, &bout);
    SCUC_TRY(rc);
    SCUC_CUDA(e3);
  }
  SCUC_CUDA(cudaGraphInstantiate(&graph_exec, g, 0));
  return SCUC_OK;
}

int Handle::solve(const scuc_solve_params& p, const double* x0_in, const double* y0_in, double* xo,
                  double* yo, double* zo, scuc_solve_info* info, double reject_kkt, bool keep_scaling) {
  using clk = std::chrono::steady_clock;
  if (!(p.tol >= 0.0) || p.check_every < 1 || p.max_iter < 1 || !(p.sigma0 > 0.0) ||
      (p.precision != SCUC_FP64 && p.precision != SCUC_MIXED) || p.power_max_iter < 1 ||
      (p.algo != SCUC_ALGO_HPR && p.algo != SCUC_ALGO_PDHG_AVG) || !(p.infeas_tol >= 0.0 && p.infeas_tol < 1.0) ||
      (p.spmv_layout != 0 && p.spmv_layout != 1) || (p.split_steps != 0 && p.split_steps != 1) ||
      !(p.polish_floor >= 0.0)) {
    set_error("invalid solve parameters");
    return SCUC_E_INVALID;
  }
  SCUC_TRY(enter());
  cudaStream_t s = work;
  const auto t0 = clk::now();
  const bool mixed = p.precision == SCUC_MIXED;
  const int64_t launch0 = nlaunch;
  SCUC_TRY(ensure_log(4096));

  // warm start in device memory
  const double *xin = nullptr, *yin = nullptr;
  if (x0_in) {
    if (p.device_ptrs) xin = x0_in;
    else {
      SCUC_CUDA(cudaMemcpyAsync(xt, x0_in, n * sizeof(double), cudaMemcpyHostToDevice, s));
      xin = xt;  // x_t and y_bar are unused until the first iteration
    }
  }
  if (y0_in) {
    if (p.device_ptrs) yin = y0_in;
    else {
      SCUC_CUDA(cudaMemcpyAsync(ybar, y0_in, m * sizeof(double), cudaMemcpyHostToDevice, s));
      yin = ybar;
    }
  }

  if (!sell_planned && p.spmv_layout == 0) {
    // sliced ELL copy of the rows of A^T that are not chunked; its values
    // are filled after every scaling
    if (m > 0 && n > 0) {
      SCUC_TRY(build_sell(rpt_plan, n, kSellMaxLen, &sT, &allocs));
      // FP32 values with 16-bit row offsets where every column allows
      SCUC_TRY(sell_values(&sT, rpt, colt, true));
    }
    // and of A's rows when A has chunked rows (the dual step of plain
    // iterations runs them beside the chunk warps); these rows are short
    // (a few entries), so a per-row record would cost more than 16-bit
    // offsets save: the 32-bit form
    if (m > 0 && n > 0 && pA.nchunk) {
      SCUC_TRY(build_sell(rp_plan, m, kSellMaxLen, &sA, &allocs));
      SCUC_TRY(sell_values(&sA, rp, col, false));
    }
    sell_planned = true;
    scaled_for = -1;  // the copies' values are filled by the next set-up
    std::vector<int>().swap(rpt_plan);
    std::vector<int>().swap(rp_plan);
  }
  const int scale_key = p.use_scaling + (mixed ? 256 : 0);
  if (!(keep_scaling && scaled_for == scale_key)) {
    scaled_for = -1;
    SCUC_TRY(setup_scaling(p.use_scaling, mixed));
    scaled_for = scale_key;
  }
  double lambda = p.lambda_in;
  int piters = 0;
  if (!(lambda > 0.0)) {
    double est = 0.0;
    SCUC_TRY(power_method(p, &est, &piters));
    lambda = p.lambda_safety * est;
    if (!(lambda > 0.0)) lambda = 1.0;
  }

  // control block: parameters and initial state
  Ctrl C{};
  SCUC_CUDA(cudaMemcpyAsync(&C, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  SCUC_CUDA(cudaStreamSynchronize(s));  // beta, gamma, bnorm, cnorm from the device
  const int64_t ce = p.check_every;
  C.tol = p.tol;
  C.sigma = p.sigma0;
  C.lambda = lambda;
  C.restart_suff = p.restart_suff;
  C.restart_nec = p.restart_nec;
  C.restart_long = p.restart_long;
  C.restart_ref = p.restart_ref;
  C.restart_metric = p.restart_metric;
  C.sigma_update = p.sigma_update;
  C.algo = p.algo;
  C.infeas_tol = p.infeas_tol;
  algo = p.algo;
  detect = p.infeas_tol > 0.0;
  use_sell = sT.nslice > 0 && p.spmv_layout == 0;
  split_steps = p.split_steps != 0;
  use_sell_dual = sA.nslice > 0 && pA.nchunk > 0 && p.spmv_layout == 0;
  C.s_step = 1.0 / (lambda * p.sigma0);
  C.polish_factor = p.polish_factor;
  C.max_iter = ((p.max_iter + ce - 1) / ce) * ce;
  C.check_every = p.check_every;
  C.polish_stall = p.polish_stall;
  C.polish_floor = p.polish_floor;
  C.log_cap = log_cap;
  C.precision = p.precision;
  C.k = 0; C.t = 0; C.iters_fp32 = 0;
  C.rho0 = 0; C.rho_prev = 0; C.best_kkt = INFINITY;
  C.first_check = 1; C.done = 0; C.status = -1; C.restart_pending = 0;
  C.reject_kkt = reject_kkt;
  C.t_start_ns = 0;
  C.time_limit_ns = (p.time_limit_s > 0.0 && p.time_limit_s < 1e9) ? (uint64_t)(p.time_limit_s * 1e9) : 0;
  C.restarts = 0; C.nlog = 0; C.fp64_phase = mixed ? 0 : 1; C.stall = 0;
  SCUC_CUDA(cudaMemcpyAsync(ctrl, &C, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
  if (p.check_every > coef_cap) {
    SCUC_TRY(alloc(&coef, 2 * (size_t)p.check_every));
    coef_cap = p.check_every;
  }
  coef_h.resize(2 * (size_t)p.check_every);
  for (int j = 0; j < p.check_every; j++) {  // weights of the first period (k = j)
    if (p.algo == SCUC_ALGO_PDHG_AVG) {      // running average
      coef_h[2 * j] = 1.0 / (double)(j + 1);
      coef_h[2 * j + 1] = (double)j / (double)(j + 1);
    } else {                                 // Halpern
      coef_h[2 * j] = 1.0 / (double)(j + 2);
      coef_h[2 * j + 1] = (double)(j + 1) / (double)(j + 2);
    }
  }
  SCUC_CUDA(cudaMemcpyAsync(coef, coef_h.data(), coef_h.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  const DevLP L = dev();
  k_init_iterates<<<grid_for(std::max(m, n)), kBlock, 0, s>>>(L, xin, yin);
  nlaunch += 1;
  SCUC_CUDA(cudaGetLastError());
  SCUC_CUDA(cudaStreamSynchronize(s));
  const auto t1 = clk::now();

  // iteration: one graph launch for the whole loop (the device decides the
  // precision of every period and when to stop), or, when profiling or
  // without graphs, one period at a time from the host
  const int64_t nper = C.max_iter / ce;
  const bool use_graph = p.use_graph && !p.profile;
  if (p.profile && (int)prof_ev.size() < 4 * p.check_every) {
    while ((int)prof_ev.size() < 4 * p.check_every) {
      cudaEvent_t e;
      SCUC_CUDA(cudaEventCreate(&e));
      prof_ev.push_back(e);
    }
  }
  double ms_p = 0.0, ms_d = 0.0, ms_p32 = 0.0, ms_d32 = 0.0;
  int64_t n_p = 0, n_d = 0, n_p32 = 0, n_d32 = 0;
  int timed_out = 0;
  if (use_graph) {
    const void* key[9] = {(const void*)(intptr_t)p.check_every, (const void*)vs32, (const void*)log_d,
                          (const void*)coef, (const void*)(intptr_t)(mixed ? 0 : 1), (const void*)(intptr_t)algo,
                          (const void*)(intptr_t)(detect ? 1 : 0), (const void*)(intptr_t)(use_sell ? 1 : 0),
                          (const void*)(intptr_t)(split_steps ? 1 : 0)};
    if (!graph_exec || memcmp(key, graph_key, sizeof(key)) != 0) {
      if (graph_exec) {
        cudaGraphExecDestroy(graph_exec);
        graph_exec = nullptr;
      }
      SCUC_TRY(build_solve_graph(p.check_every, mixed ? 0 : 1));
      memcpy(graph_key, key, sizeof(key));
    }
    SCUC_CUDA(cudaGraphLaunch(graph_exec, s));
    SCUC_CUDA(cudaStreamSynchronize(s));
    SCUC_CUDA(cudaMemcpyAsync(&C, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaStreamSynchronize(s));
    nlaunch += ((C.t + ce - 1) / ce) * (period_kernels(p.check_every) + 1);
  } else {
    int phase64 = mixed ? 0 : 1;  // phase of the next period (the host waits for every period)
    for (int64_t per = 0; per < nper; per++) {
      SCUC_TRY(launch_period(p.check_every, p.profile != 0, phase64 != 0));
      SCUC_CUDA(cudaMemcpyAsync(ctrl_h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
      SCUC_CUDA(cudaEventRecord(ev_slot[0], s));
      SCUC_CUDA(cudaEventSynchronize(ev_slot[0]));
      if (p.profile) {
        for (int j = 0; j < p.check_every; j++) {
          float a = 0.f, b = 0.f;
          SCUC_CUDA(cudaEventElapsedTime(&a, prof_ev[4 * j + 0], prof_ev[4 * j + 1]));
          SCUC_CUDA(cudaEventElapsedTime(&b, prof_ev[4 * j + 2], prof_ev[4 * j + 3]));
          ms_p += a; ms_d += b;
          if (!phase64) { ms_p32 += a; ms_d32 += b; }
        }
        n_p += p.check_every; n_d += p.check_every;
        if (!phase64) { n_p32 += p.check_every; n_d32 += p.check_every; }
      }
      phase64 = ctrl_h[0].fp64_phase;
      if (ctrl_h[0].done) break;
      const double el = std::chrono::duration<double>(clk::now() - t0).count();
      if (el > p.time_limit_s) { timed_out = 1; break; }
    }
  }
  SCUC_CUDA(cudaStreamSynchronize(s));
  SCUC_CUDA(cudaMemcpyAsync(&C, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  SCUC_CUDA(cudaStreamSynchronize(s));
  const auto t2 = clk::now();

  // outputs (unscaled)
  double *dxo = xo, *dyo = yo, *dzo = zo;
  if (!p.device_ptrs) {
    dxo = xo ? xt : nullptr;    // scratch: xt, wv (n), uv (m)
    dzo = zo ? wv : nullptr;
    dyo = yo ? uv : nullptr;
  }
  k_finalize<<<grid_for(std::max(m, n)), kBlock, 0, s>>>(L, dxo, dyo, dzo);
  nlaunch += 1;
  SCUC_CUDA(cudaGetLastError());
  if (!p.device_ptrs) {
    if (xo) SCUC_CUDA(cudaMemcpyAsync(xo, dxo, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (yo) SCUC_CUDA(cudaMemcpyAsync(yo, dyo, m * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (zo) SCUC_CUDA(cudaMemcpyAsync(zo, dzo, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  last_nlog = std::min(C.nlog, log_cap);
  SCUC_CUDA(cudaStreamSynchronize(s));
  if (info) {
    memset(info, 0, sizeof(*info));
    info->status = timed_out && !C.done ? SCUC_ST_TIME_LIMIT : (C.status < 0 ? SCUC_ST_ITER_LIMIT : C.status);
    info->restarts = C.restarts;
    info->iters = C.t;
    info->iters_fp32 = C.iters_fp32;
    info->power_iters = piters;
    info->nlog = last_nlog;
    info->kkt = C.kkt; info->rp = C.rp; info->rd = C.rd; info->gap = C.gap;
    info->pobj = C.pobj; info->dobj = C.dobj;
    info->lambda = C.lambda; info->sigma = C.sigma; info->beta = C.beta; info->gamma = C.gamma;
    info->setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    info->solve_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
    info->ms_dual_spmv = ms_d; info->ms_primal_spmv = ms_p;
    info->n_dual_spmv = n_d; info->n_primal_spmv = n_p;
    info->ms_dual_spmv_f32 = ms_d32; info->ms_primal_spmv_f32 = ms_p32;
    info->n_dual_spmv_f32 = n_d32; info->n_primal_spmv_f32 = n_p32;
    info->launches = nlaunch - launch0;
  }
  return leave();
}

int Handle::matvec(int transpose, const double* in, double* out) {
  SCUC_TRY(enter());
  cudaStream_t s = work;
  const Partition& P = transpose ? pT : pA;
  const int* r = transpose ? rpt : rp;
  const int* c = transpose ? colt : col;
  const double* v = transpose ? valt : val;
  if (P.nchunk) k_chunk_sums<double><<<P.nchunkblk, kBlock, 0, s>>>(c, v, in, P);
  if (P.nblk) k_spmv_plain<<<P.nblk, kBlock, P.smem, s>>>(r, c, v, in, P, out);
  SCUC_CUDA(cudaGetLastError());
  SCUC_CUDA(cudaStreamSynchronize(s));
  return leave();
}

}  // namespace scuc

// ===========================================================================
// C ABI
// ===========================================================================
using scuc::Handle;

extern "C" {

void scuc_default_params(scuc_solve_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->tol = 1e-4;
  p->max_iter = 1000000;
  p->time_limit_s = 3600.0;
  p->check_every = 64;
  p->precision = SCUC_FP64;
  p->use_scaling = 1;
  p->sigma0 = 1.0;
  p->lambda_in = 0.0;
  p->lambda_safety = 1.01;
  p->power_max_iter = 500;
  p->power_tol = 1e-4;
  p->power_seed = 0x5EED;
  p->restart_suff = 0.2;
  p->restart_nec = 0.8;
  p->restart_long = 0.2;
  p->polish_factor = 1.0;
  p->polish_stall = 200;
  p->polish_floor = 1e-6;
  p->use_graph = 1;
  p->profile = 0;
  p->device_ptrs = 0;
  p->restart_ref = 0;
  p->restart_metric = 0;
  p->sigma_update = 1;
  p->algo = SCUC_ALGO_HPR;
  p->infeas_tol = 0.0;
}

static int sense_to_box(int32_t m, const char* sense, const double* rhs, const double* range,
                        std::vector<double>& lo, std::vector<double>& hi) {
  lo.assign(m, -INFINITY);
  hi.assign(m, INFINITY);
  if (m > 0 && (!sense || !rhs)) {
    scuc::set_error("sense and rhs are required");
    return SCUC_E_INVALID;
  }
  for (int32_t i = 0; i < m; i++) {
    switch (sense[i]) {
      case 'G': lo[i] = rhs[i]; break;
      case 'L': hi[i] = rhs[i]; break;
      case 'E': lo[i] = rhs[i]; hi[i] = rhs[i]; break;
      case 'R':
        if (!range || !(range[i] >= 0.0)) {
          scuc::set_error("row %d: 'R' needs range >= 0", i);
          return SCUC_E_INVALID;
        }
        lo[i] = rhs[i];
        hi[i] = rhs[i] + range[i];
        break;
      default:
        scuc::set_error("row %d: unknown sense", i);
        return SCUC_E_INVALID;
    }
  }
  return SCUC_OK;
}

int scuc_lp_create(scuc_lp** out, int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                   const int32_t* col, const double* val, const double* c, const double* xl,
                   const double* xu, const char* sense, const double* rhs, const double* range,
                   void* cuda_stream) {
  if (!out) { scuc::set_error("out is NULL"); return SCUC_E_INVALID; }
  if (m < 0) { scuc::set_error("m < 0"); return SCUC_E_INVALID; }
  std::vector<double> lo, hi;
  SCUC_TRY(sense_to_box(m, sense, rhs, range, lo, hi));
  return scuc_lp_create_box(out, m, n, nnz, row_ptr, col, val, c, xl, xu, lo.data(), hi.data(),
                            cuda_stream);
}

int scuc_lp_create_box(scuc_lp** out, int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                       const int32_t* col, const double* val, const double* c, const double* xl,
                       const double* xu, const double* lo, const double* hi, void* cuda_stream) {
  if (!out) { scuc::set_error("out is NULL"); return SCUC_E_INVALID; }
  *out = nullptr;
  Handle* h = nullptr;
  SCUC_TRY(scuc::create_handle(&h, m, n, nnz, row_ptr, col, val, c, xl, xu, lo, hi, cuda_stream));
  *out = new scuc_lp{h};
  return SCUC_OK;
}

int scuc_lp_layout(const scuc_lp* lp, int64_t* out) {
  if (!lp || !out) { scuc::set_error("null handle or output"); return SCUC_E_INVALID; }
  const Handle* h = lp->h;
  out[0] = (int64_t)h->n16_h[0];
  out[1] = h->pA.nchunk_ent - out[0];
  out[2] = h->sA.nent;
  out[3] = h->sT.compressed ? h->sT.npair * 64 : h->sT.nent;
  out[4] = h->sT.compressed;
  out[5] = (int64_t)h->sT.nslice * 32;
  out[6] = (int64_t)h->n16_h[1];
  out[7] = h->pT.nchunk_ent - out[6];
  return SCUC_OK;
}

int scuc_lp_set_index16(scuc_lp* lp, int32_t on) {
  if (!lp) { scuc::set_error("null handle"); return SCUC_E_INVALID; }
  Handle* h = lp->h;
  if (on != 0 && on != 1) { scuc::set_error("index16 must be 0 or 1"); return SCUC_E_INVALID; }
  if (h->vs32 || h->sell_planned) {
    scuc::set_error("index16 is set before the handle's first solve");
    return SCUC_E_INVALID;
  }
  h->index16 = on != 0;
  return SCUC_OK;
}

int scuc_lp_dims(const scuc_lp* lp, int32_t* m, int32_t* n, int64_t* nnz) {
  if (!lp) { scuc::set_error("null handle"); return SCUC_E_INVALID; }
  if (m) *m = lp->h->m;
  if (n) *n = lp->h->n;
  if (nnz) *nnz = lp->h->nnz;
  return SCUC_OK;
}

int scuc_lp_solve(scuc_lp* lp, const scuc_solve_params* p, const double* x0, const double* y0,
                  double* x_out, double* y_out, double* z_out, scuc_solve_info* info) {
  if (!lp) { scuc::set_error("null handle"); return SCUC_E_INVALID; }
  scuc_solve_params d;
  if (!p) { scuc_default_params(&d); p = &d; }
  return lp->h->solve(*p, x0, y0, x_out, y_out, z_out, info);
}

int scuc_lp_get_log(const scuc_lp* lp, scuc_check_log* out, int32_t cap, int32_t* count) {
  if (!lp || (!out && cap > 0)) { scuc::set_error("null argument"); return SCUC_E_INVALID; }
  const Handle* h = lp->h;
  int k = std::min(cap, h->last_nlog);
  if (k > 0) SCUC_CUDA(cudaMemcpy(out, h->log_d, k * sizeof(scuc_check_log), cudaMemcpyDeviceToHost));
  if (count) *count = k;
  return SCUC_OK;
}

int scuc_lp_matvec(scuc_lp* lp, int32_t transpose, const double* in_dev, double* out_dev) {
  if (!lp || !in_dev || !out_dev) { scuc::set_error("null argument"); return SCUC_E_INVALID; }
  return lp->h->matvec(transpose, in_dev, out_dev);
}

int scuc_lp_solve_batch(scuc_lp* const* lps, int32_t count, const scuc_solve_params* p,
                        double* const* x_out, double* const* y_out, double* const* z_out,
                        scuc_solve_info* infos, scuc_batch_info* binfo) {
  if (!lps || count < 0 || (count > 0 && !infos)) {
    scuc::set_error("scuc_lp_solve_batch: null argument");
    return SCUC_E_INVALID;
  }
  if (count == 0) return SCUC_OK;
  std::vector<Handle*> H(count);
  for (int32_t i = 0; i < count; i++) {
    if (!lps[i] || !lps[i]->h) {
      scuc::set_error("scuc_lp_solve_batch: LP %d is null", i);
      return SCUC_E_INVALID;
    }
    H[i] = lps[i]->h;
  }
  scuc_solve_params q;
  if (p) q = *p;
  else scuc_default_params(&q);
  return scuc::solve_batch(H.data(), count, q, x_out, y_out, z_out, infos, binfo);
}

void scuc_lp_destroy(scuc_lp* lp) {
  if (!lp) return;
  delete lp->h;
  delete lp;
}

const char* scuc_last_error(void) { return scuc::g_err.c_str(); }

}  // extern "C"
