// Many LP relaxations solved together (scuc_lp_solve_batch): the LPs are
// laid out as one block-diagonal LP and every iteration of Eq. 9 runs as one
// launch over all of them, so small LPs (a few thousand rows each) fill the
// GPU together instead of each leaving most of it idle.  Every LP keeps its
// own scaling, lambda, sigma, Halpern counter, restarts, precision phase and
// stop decision: the kernels find the LP of a block in a per-block table,
// the decide kernel runs one block per LP, and blocks of LPs that have
// stopped return at once.  The SpMV partitions never let a block span two
// LPs; their shape (entries per thread of list rows, shortest staged run)
// is chosen by timing candidate partitions on the batch.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "lp.h"
#include "setup_kernels.cuh"

namespace scuc {
namespace {

__global__ void k_add_offset(int* __restrict__ dst, const int* __restrict__ src, int64_t count, int add) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += step) dst[e] = src[e] + add;
}

template <typename VT>
struct TuneEpi {
  VT* out;
  __device__ void load(int) {}
  __device__ void row(int r, VT a) { out[r] = a; }
};

template <typename VT>
__global__ void __launch_bounds__(kBlock) k_spmv_tune(const int* __restrict__ rp, const int* __restrict__ col,
                                                      const VT* __restrict__ val, const VT* __restrict__ in,
                                                      Partition part, VT* __restrict__ out) {
  extern __shared__ __align__(128) unsigned char smem[];
  TuneEpi<VT> epi{out};
  spmv_block<VT>(rp, col, val, in, part, smem, epi);
}

int grid_b(int64_t n) {
  const int64_t g = (n + kBlock - 1) / kBlock;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 148 * 16));
}

struct Batch {
  int nlp = 0, m = 0, n = 0;
  int64_t nnz = 0;
  bool mixed = false;
  cudaStream_t s = nullptr;
  std::vector<void*> allocs;
  int *rp = nullptr, *col = nullptr, *rpt = nullptr, *colt = nullptr;
  double *vs = nullptr, *vst = nullptr;
  float *vs32 = nullptr, *vst32 = nullptr;
  double *cs = nullptr, *xls = nullptr, *xus = nullptr, *los = nullptr, *his = nullptr, *Dr = nullptr,
         *Dc = nullptr;
  double *x = nullptr, *x0 = nullptr, *xt = nullptr, *xbar = nullptr, *zbar = nullptr;
  double *y = nullptr, *y0 = nullptr, *ybar = nullptr, *qchk = nullptr, *dychk = nullptr;
  float *xt32 = nullptr, *y32 = nullptr;
  double *partP = nullptr, *partD = nullptr, *partRA = nullptr, *partRT = nullptr;
  double* gsum = nullptr;
  float* gsum32 = nullptr;
  int epi_gx = 1;
  double *xo = nullptr, *yo = nullptr, *zo = nullptr;
  Ctrl* ctrl = nullptr;
  Ctrl* ctrl_h = nullptr;  // pinned, two slots of nlp
  double* coef = nullptr;
  scuc_check_log* log = nullptr;
  int log_cap = 0, coef_stride = 0;
  int *blkA = nullptr, *blkT = nullptr, *ablk0 = nullptr, *tblk0 = nullptr, *row0 = nullptr, *col0 = nullptr;
  Partition pA, pT;
  std::vector<int> row0_h, col0_h;
  std::vector<int64_t> nnz0_h;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t ev_slot[2] = {nullptr, nullptr};

  ~Batch() {
    if (s) cudaStreamSynchronize(s);
    if (graph) cudaGraphExecDestroy(graph);
    for (auto& e : ev_slot)
      if (e) cudaEventDestroy(e);
    free_partition(&pA);
    free_partition(&pT);
    for (void* p : allocs) dev_free(p);
    if (ctrl_h) cudaFreeHost(ctrl_h);
    if (s) cudaStreamDestroy(s);
  }
  template <typename T>
  int alloc(T** p, size_t count) {
    void* q = nullptr;
    SCUC_TRY(dev_alloc_bytes(&q, std::max<size_t>(count, 1) * sizeof(T)));
    allocs.push_back(q);
    *p = static_cast<T*>(q);
    return SCUC_OK;
  }
  DevLP dev() const {
    DevLP L;
    L.m = m; L.n = n;
    L.rp = rp; L.col = col; L.rpt = rpt; L.colt = colt;
    L.vs = vs; L.vst = vst; L.vs32 = vs32; L.vst32 = vst32; L.val = nullptr; L.valt = nullptr;
    L.c = cs; L.xl = xls; L.xu = xus; L.lo = los; L.hi = his; L.Dr = Dr; L.Dc = Dc;
    L.x = x; L.x0 = x0; L.xt = xt; L.xbar = xbar; L.zbar = zbar; L.y = y; L.y0 = y0; L.ybar = ybar;
    L.xt32 = xt32; L.y32 = y32;
    L.qchk = qchk; L.dychk = dychk;
    L.dxchk = nullptr;  // no infeasibility detection in batches
    L.coef = coef; L.coef_w = coef;
    L.partP = partP; L.partD = partD; L.partRA = partRA; L.partRT = partRT;
    L.gsum = gsum;
    L.gsum32 = gsum32;
    L.epi_gx = epi_gx;
    L.pA = pA; L.pT = pT;
    L.ctrl = ctrl; L.log = log;
    L.nlp = nlp;
    L.blkA = blkA; L.blkT = blkT; L.ablk0 = ablk0; L.tblk0 = tblk0; L.row0 = row0; L.col0 = col0;
    L.coef_stride = coef_stride;
    L.log_stride = log_cap;
    return L;
  }
};

// Partition of the block-diagonal matrix: each LP's rows planned alone (no
// chunked rows), then merged class by class with row and entry offsets; an
// LP's rows of one class are padded to whole blocks, so no block spans two
// LPs.  Blocks write their partial sums LP by LP (slot table), so each LP's
// partials form one range for the decide kernel.
void plan_batch(const std::vector<std::vector<int>>& rps, const std::vector<int>& off,
                const std::vector<int64_t>& eoff, const PartShape& shape, PartPlan* plan,
                std::vector<int>* blk_lp, std::vector<int>* blk0) {
  const int nlp = (int)rps.size();
  std::vector<PartPlan> one(nlp);
  for (int b = 0; b < nlp; b++) plan_partition(rps[b], (int)rps[b].size() - 1, shape, false, &one[b]);
  *plan = PartPlan{};
  plan->chunk_ptr.assign(1, 0);
  blk_lp->clear();
  for (int k = 0; k < 4; k++) {
    const int per = kBlock >> (5 - k);
    plan->cls_row[k] = (int)plan->listx.size();
    plan->cls_blk[k] = (int)blk_lp->size();
    for (int b = 0; b < nlp; b++) {
      const int n0 = one[b].cls_row[k], n1 = one[b].cls_row[k + 1];
      if (n1 == n0) continue;
      for (int i = n0; i < n1; i++) {
        int4 e = one[b].listx[i];
        plan->listx.push_back(make_int4(e.x + off[b], e.y + (int)eoff[b], e.z + (int)eoff[b], 0));
      }
      const int nb = (n1 - n0 + per - 1) / per;
      for (int q = (n1 - n0); q < nb * per; q++) plan->listx.push_back(make_int4(-1, 0, 0, 0));
      for (int q = 0; q < nb; q++) blk_lp->push_back(b);
    }
  }
  plan->cls_row[4] = (int)plan->listx.size();
  plan->cls_blk[4] = (int)blk_lp->size();
  for (int b = 0; b < nlp; b++)
    for (int4 d : one[b].desc) {
      plan->desc.push_back(make_int4(d.x + off[b], d.y + (int)eoff[b], d.z + (int)eoff[b], d.w));
      blk_lp->push_back(b);
    }
  // slots: blocks ordered by LP (stable)
  const int nblk = (int)blk_lp->size();
  std::vector<int> cnt(nlp + 1, 0);
  for (int q : *blk_lp) cnt[q + 1]++;
  for (int b = 0; b < nlp; b++) cnt[b + 1] += cnt[b];
  *blk0 = cnt;
  plan->slot.assign(nblk, 0);
  std::vector<int> next(cnt.begin(), cnt.end() - 1);
  for (int q = 0; q < nblk; q++) plan->slot[q] = next[(*blk_lp)[q]]++;
}

// Shapes chosen for earlier batches, keyed by precision and the sizes of
// the batch's LPs (m, n, nnz of each, in order).
std::mutex g_shape_mu;
std::map<std::vector<int64_t>, std::pair<PartShape, PartShape>> g_shapes;

bool tuned_shapes(const std::vector<int64_t>& key, PartShape* a, PartShape* t) {
  std::lock_guard<std::mutex> lock(g_shape_mu);
  auto it = g_shapes.find(key);
  if (it == g_shapes.end()) return false;
  *a = it->second.first;
  *t = it->second.second;
  return true;
}

void remember_shapes(const std::vector<int64_t>& key, const PartShape& a, const PartShape& t) {
  std::lock_guard<std::mutex> lock(g_shape_mu);
  g_shapes[key] = std::make_pair(a, t);
}

// Time one SpMV over the candidate partition (median of three launches).
template <typename VT>
int time_spmv(const int* rp, const int* col, const VT* val, const VT* in, VT* out, const Partition& P,
              cudaStream_t s, float* ms) {
  cudaEvent_t e[4];
  for (auto& q : e) SCUC_CUDA(cudaEventCreate(&q));
  float t[3];
  k_spmv_tune<VT><<<P.nblk, kBlock, P.smem, s>>>(rp, col, val, in, P, out);  // warm-up
  for (int i = 0; i < 3; i++) {
    SCUC_CUDA(cudaEventRecord(e[0], s));
    k_spmv_tune<VT><<<P.nblk, kBlock, P.smem, s>>>(rp, col, val, in, P, out);
    SCUC_CUDA(cudaEventRecord(e[1], s));
    SCUC_CUDA(cudaEventSynchronize(e[1]));
    SCUC_CUDA(cudaEventElapsedTime(&t[i], e[0], e[1]));
  }
  SCUC_CUDA(cudaGetLastError());
  for (auto& q : e) cudaEventDestroy(q);
  std::sort(t, t + 3);
  *ms = t[1];
  return SCUC_OK;
}

// Choose the shape of one matrix's partition (A or A^T of the batch) and
// upload it: blk / blk0 get the per-block LP table and LP block offsets.
int tune_partition(Batch& B, bool transpose, const std::vector<std::vector<int>>& rps,
                   const std::vector<int>& off, const std::vector<int64_t>& eoff, bool autotune, Partition* P,
                   int** blk, int** blk0, PartShape* chosen, int* ncand, const PartShape* given) {
  std::vector<PartShape> cands;
  if (given) {
    cands.push_back(*given);
  } else if (autotune) {
    for (int ept : {8, 12, 16})
      for (int run : {16, 64}) {
        PartShape sh;
        sh.ept = ept;
        sh.min_run = run;
        cands.push_back(sh);
      }
  } else {
    cands.push_back(PartShape{});
  }
  *ncand = (int)cands.size();
  const int rows = transpose ? B.n : B.m;
  const int* rp = transpose ? B.rpt : B.rp;
  const int* col = transpose ? B.colt : B.col;
  PartPlan plan;
  std::vector<int> lp, b0;
  float best = -1.f;
  PartShape best_sh = cands[0];
  if (cands.size() > 1) {
    for (const PartShape& sh : cands) {
      plan_batch(rps, off, eoff, sh, &plan, &lp, &b0);
      Partition T;
      SCUC_TRY(upload_partition(plan, &T));
      float ms = 0.f;
      int rc = SCUC_OK;
      if (T.nblk == 0) {
        // nothing to time
      } else if (B.mixed) {
        const float* in = transpose ? B.y32 : B.xt32;
        float* out = transpose ? B.xt32 : B.y32;  // the other shadow: sized for the output
        rc = time_spmv<float>(rp, col, transpose ? B.vst32 : B.vs32, in, out, T, B.s, &ms);
      } else {
        const double* in = transpose ? B.ybar : B.xbar;
        double* out = transpose ? B.zbar : B.qchk;
        rc = time_spmv<double>(rp, col, transpose ? B.vst : B.vs, in, out, T, B.s, &ms);
      }
      free_partition(&T);
      SCUC_TRY(rc);
      if (best < 0.f || ms < best) {
        best = ms;
        best_sh = sh;
      }
    }
  }
  (void)rows;
  plan_batch(rps, off, eoff, best_sh, &plan, &lp, &b0);
  SCUC_TRY(upload_partition(plan, P));
  SCUC_TRY(B.alloc(blk, lp.size()));
  SCUC_TRY(B.alloc(blk0, b0.size()));
  if (!lp.empty()) SCUC_CUDA(cudaMemcpy(*blk, lp.data(), lp.size() * sizeof(int), cudaMemcpyHostToDevice));
  SCUC_CUDA(cudaMemcpy(*blk0, b0.data(), b0.size() * sizeof(int), cudaMemcpyHostToDevice));
  *chosen = best_sh;
  return SCUC_OK;
}

// One period over all LPs (runtime precision: each LP's own phase).
int launch_batch_period(Batch& B, cudaStream_t s, int check_every, int ga) {
  const DevLP L = B.dev();
  k_anchor<<<dim3(ga, B.nlp), kBlock, 0, s>>>(L);
  for (int j = 0; j < check_every; j++) {
    const bool chk = (j == check_every - 1);
    if (B.pT.nblk) k_primal_sum<kPrecRuntime><<<B.pT.nblk, kBlock, B.pT.smem, s>>>(L);
    if (chk) k_primal_epi<true, kPrecRuntime><<<dim3(B.epi_gx, B.nlp), kBlock, 0, s>>>(L, j);
    else k_primal_epi<false, kPrecRuntime><<<dim3(B.epi_gx, B.nlp), kBlock, 0, s>>>(L, j);
    if (B.pA.nblk) {
      if (chk) k_dual<true, kPrecRuntime><<<B.pA.nblk, kBlock, B.pA.smem, s>>>(L, j);
      else k_dual<false, kPrecRuntime><<<B.pA.nblk, kBlock, B.pA.smem, s>>>(L, j);
    }
  }
  if (B.pA.nblk) k_res_primal<<<B.pA.nblk, kBlock, B.pA.smem, s>>>(L);
  if (B.pT.nblk) k_res_dual<false><<<B.pT.nblk, kBlock, B.pT.smem, s>>>(L);
  k_decide<<<B.nlp, kDecideThreads, 0, s>>>(L, check_every);
  SCUC_CUDA(cudaGetLastError());
  return SCUC_OK;
}

int64_t period_launches(const Batch& B, int ce) {
  return 2 + (int64_t)ce * ((B.pT.nblk ? 1 : 0) + (B.pA.nblk ? 1 : 0) + 1) + (B.pA.nblk ? 1 : 0) +
         (B.pT.nblk ? 1 : 0);
}

// The batch's iteration as one graph: WHILE (some LP runs) { period; conditions }.
int build_batch_graph(Batch& B, int check_every, int ga) {
  cudaGraph_t g = nullptr;
  SCUC_CUDA(cudaGraphCreate(&g, 0));
  struct GraphGuard {
    cudaGraph_t g;
    ~GraphGuard() { if (g) cudaGraphDestroy(g); }
  } guard{g};
  cudaGraphConditionalHandle hloop;
  SCUC_CUDA(cudaGraphConditionalHandleCreate(&hloop, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hloop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  SCUC_CUDA(cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp));
  SCUC_CUDA(cudaStreamBeginCaptureToGraph(B.s, wp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
  int rc = launch_batch_period(B, B.s, check_every, ga);
  if (rc == SCUC_OK) k_loop_cond<<<1, kDecideThreads, 0, B.s>>>(B.dev(), hloop, hloop, 0);
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(B.s, &out);
  SCUC_TRY(rc);
  SCUC_CUDA(e);
  SCUC_CUDA(cudaGraphInstantiate(&B.graph, g, 0));
  return SCUC_OK;
}

}  // namespace

int solve_batch(Handle* const* H, int nlp, const scuc_solve_params& p, double* const* xo, double* const* yo,
                double* const* zo, scuc_solve_info* infos, scuc_batch_info* bi) {
  using clk = std::chrono::steady_clock;
  if (!(p.tol >= 0.0) || p.check_every < 1 || p.max_iter < 1 || !(p.sigma0 > 0.0) ||
      (p.precision != SCUC_FP64 && p.precision != SCUC_MIXED) || p.power_max_iter < 1) {
    set_error("invalid solve parameters");
    return SCUC_E_INVALID;
  }
  if (p.algo != SCUC_ALGO_HPR || p.infeas_tol != 0.0) {
    set_error("scuc_lp_solve_batch: batches run SCUC_ALGO_HPR without infeasibility detection");
    return SCUC_E_INVALID;
  }
  if (nlp > 65535) {
    set_error("scuc_lp_solve_batch: at most 65535 LPs per batch");
    return SCUC_E_INVALID;
  }
  const int device = H[0]->device;
  for (int b = 0; b < nlp; b++) {
    if (H[b]->device != device) {
      set_error("scuc_lp_solve_batch: LP %d lives on device %d, LP 0 on device %d", b, H[b]->device, device);
      return SCUC_E_INVALID;
    }
    for (int q = 0; q < b; q++)
      if (H[q] == H[b]) {
        set_error("scuc_lp_solve_batch: LP %d appears twice (also as LP %d)", b, q);
        return SCUC_E_INVALID;
      }
  }
  const bool autotune = bi ? bi->autotune != 0 : true;
  const auto t0 = clk::now();
  const bool mixed = p.precision == SCUC_MIXED;
  int64_t launches = 0;

  // 1. scaling and lambda of every LP, on its own handle and stream (Sec.
  // 3.A, Eq. 9): every LP's scaling and power-method rounds are queued
  // before any is waited for, so the LPs' small launches overlap
  std::vector<double> lam(nlp, p.lambda_in);
  std::vector<int> piters(nlp, 0);
  std::vector<Ctrl> C(nlp);
  std::vector<int64_t> l0(nlp);
  const bool power = !(p.lambda_in > 0.0);
  for (int b = 0; b < nlp; b++) {
    Handle& h = *H[b];
    SCUC_TRY(h.enter());
    l0[b] = h.nlaunch;
    SCUC_TRY(h.setup_scaling(p.use_scaling, mixed));
    if (power) SCUC_TRY(h.power_start(p));
  }
  std::vector<char> pdone(nlp, power ? 0 : 1);
  for (bool all = !power; !all;) {
    for (int b = 0; b < nlp; b++)
      if (!pdone[b]) SCUC_TRY(H[b]->power_round(p));
    all = true;
    for (int b = 0; b < nlp; b++) {
      if (pdone[b]) continue;
      bool d = false;
      double est = 0.0;
      SCUC_TRY(H[b]->power_poll(p, &d, &est, &piters[b]));
      if (d) {
        pdone[b] = 1;
        lam[b] = p.lambda_safety * est;
        if (!(lam[b] > 0.0)) lam[b] = 1.0;
      } else {
        all = false;
      }
    }
  }
  for (int b = 0; b < nlp; b++) {
    Handle& h = *H[b];
    SCUC_CUDA(cudaMemcpyAsync(&C[b], h.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h.work));
    launches += h.nlaunch - l0[b];
  }
  for (int b = 0; b < nlp; b++) SCUC_CUDA(cudaStreamSynchronize(H[b]->work));
  const auto ts1 = clk::now();

  // 2. the block-diagonal LP
  Batch B;
  B.nlp = nlp;
  B.mixed = mixed;
  SCUC_CUDA(cudaSetDevice(device));
  SCUC_CUDA(cudaStreamCreateWithFlags(&B.s, cudaStreamNonBlocking));
  SCUC_CUDA(cudaEventCreateWithFlags(&B.ev_slot[0], cudaEventDisableTiming));
  SCUC_CUDA(cudaEventCreateWithFlags(&B.ev_slot[1], cudaEventDisableTiming));
  B.row0_h.assign(nlp + 1, 0);
  B.col0_h.assign(nlp + 1, 0);
  B.nnz0_h.assign(nlp + 1, 0);
  int64_t mt = 0, nt = 0, zt = 0;
  for (int b = 0; b < nlp; b++) {
    mt += H[b]->m;
    nt += H[b]->n;
    zt += H[b]->nnz;
    if (mt >= INT_MAX || nt >= INT_MAX || zt >= INT_MAX) {
      set_error("scuc_lp_solve_batch: the batch exceeds 2^31 - 1 rows, columns or nonzeros");
      return SCUC_E_INVALID;
    }
    B.row0_h[b + 1] = (int)mt;
    B.col0_h[b + 1] = (int)nt;
    B.nnz0_h[b + 1] = zt;
  }
  B.m = (int)mt;
  B.n = (int)nt;
  B.nnz = zt;
  const int m = B.m, n = B.n;
  const int64_t nnz = B.nnz;
  SCUC_TRY(B.alloc(&B.rp, m + 1));
  SCUC_TRY(B.alloc(&B.col, nnz));
  SCUC_TRY(B.alloc(&B.rpt, n + 1));
  SCUC_TRY(B.alloc(&B.colt, nnz));
  SCUC_TRY(B.alloc(&B.vs, nnz));
  SCUC_TRY(B.alloc(&B.vst, nnz));
  if (mixed) {
    SCUC_TRY(B.alloc(&B.vs32, nnz));
    SCUC_TRY(B.alloc(&B.vst32, nnz));
  }
  for (double** a : {&B.cs, &B.xls, &B.xus, &B.Dc, &B.x, &B.x0, &B.xt, &B.xbar, &B.zbar, &B.xo, &B.zo})
    SCUC_TRY(B.alloc(a, n));
  for (double** a : {&B.los, &B.his, &B.Dr, &B.y, &B.y0, &B.ybar, &B.qchk, &B.dychk, &B.yo})
    SCUC_TRY(B.alloc(a, m));
  SCUC_TRY(B.alloc(&B.xt32, n));
  SCUC_TRY(B.alloc(&B.y32, m));
  cudaStream_t s = B.s;
  SCUC_CUDA(cudaMemsetAsync(B.xt32, 0, (size_t)n * sizeof(float), s));
  SCUC_CUDA(cudaMemsetAsync(B.y32, 0, (size_t)m * sizeof(float), s));
  SCUC_CUDA(cudaMemsetAsync(B.xbar, 0, (size_t)n * sizeof(double), s));
  SCUC_CUDA(cudaMemsetAsync(B.zbar, 0, (size_t)n * sizeof(double), s));
  SCUC_CUDA(cudaMemsetAsync(B.ybar, 0, (size_t)m * sizeof(double), s));
  std::vector<std::vector<int>> rps(nlp), rpts(nlp);
  for (int b = 0; b < nlp; b++) {
    const Handle& h = *H[b];
    const int r0 = B.row0_h[b], c0 = B.col0_h[b];
    const int64_t z0 = B.nnz0_h[b];
    auto cp = [&](void* dst, const void* src, size_t bytes) {
      return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s) : cudaSuccess;
    };
    if (h.m) k_add_offset<<<grid_b(h.m), kBlock, 0, s>>>(B.rp + r0, h.rp, h.m, (int)z0);
    if (h.n) k_add_offset<<<grid_b(h.n), kBlock, 0, s>>>(B.rpt + c0, h.rpt, h.n, (int)z0);
    if (h.nnz) {
      k_add_offset<<<grid_b(h.nnz), kBlock, 0, s>>>(B.col + z0, h.col, h.nnz, c0);
      k_add_offset<<<grid_b(h.nnz), kBlock, 0, s>>>(B.colt + z0, h.colt, h.nnz, r0);
    }
    launches += (h.m ? 1 : 0) + (h.n ? 1 : 0) + (h.nnz ? 2 : 0);
    SCUC_CUDA(cudaGetLastError());
    SCUC_CUDA(cp(B.vs + z0, h.vs, h.nnz * sizeof(double)));
    SCUC_CUDA(cp(B.vst + z0, h.vst, h.nnz * sizeof(double)));
    if (mixed) {
      SCUC_CUDA(cp(B.vs32 + z0, h.vs32, h.nnz * sizeof(float)));
      SCUC_CUDA(cp(B.vst32 + z0, h.vst32, h.nnz * sizeof(float)));
    }
    const size_t nb = (size_t)h.n * sizeof(double), mb = (size_t)h.m * sizeof(double);
    SCUC_CUDA(cp(B.cs + c0, h.cs, nb));
    SCUC_CUDA(cp(B.xls + c0, h.xls, nb));
    SCUC_CUDA(cp(B.xus + c0, h.xus, nb));
    SCUC_CUDA(cp(B.Dc + c0, h.Dc, nb));
    SCUC_CUDA(cp(B.los + r0, h.los, mb));
    SCUC_CUDA(cp(B.his + r0, h.his, mb));
    SCUC_CUDA(cp(B.Dr + r0, h.Dr, mb));
    rps[b].resize(h.m + 1);
    rpts[b].resize(h.n + 1);
    SCUC_CUDA(cudaMemcpyAsync(rps[b].data(), h.rp, (h.m + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaMemcpyAsync(rpts[b].data(), h.rpt, (h.n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  const int tot = (int)nnz;
  SCUC_CUDA(cudaMemcpyAsync(B.rp + m, &tot, sizeof(int), cudaMemcpyHostToDevice, s));
  SCUC_CUDA(cudaMemcpyAsync(B.rpt + n, &tot, sizeof(int), cudaMemcpyHostToDevice, s));
  SCUC_TRY(B.alloc(&B.row0, nlp + 1));
  SCUC_TRY(B.alloc(&B.col0, nlp + 1));
  SCUC_CUDA(cudaMemcpyAsync(B.row0, B.row0_h.data(), (nlp + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  SCUC_CUDA(cudaMemcpyAsync(B.col0, B.col0_h.data(), (nlp + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  SCUC_CUDA(cudaStreamSynchronize(s));

  // 3. partitions (autotuned shapes; a batch of the same LP sizes and
  // precision reuses the shapes tuned for it before)
  const auto tt0 = clk::now();
  PartShape shA, shT;
  int ncA = 0, ncT = 0;
  std::vector<int64_t> key;
  key.push_back(mixed ? 1 : 0);
  key.push_back(nlp);
  for (int b = 0; b < nlp; b++) {
    key.push_back(H[b]->m);
    key.push_back(H[b]->n);
    key.push_back(H[b]->nnz);
  }
  const bool cached = autotune && tuned_shapes(key, &shA, &shT);
  SCUC_TRY(tune_partition(B, false, rps, B.row0_h, B.nnz0_h, autotune && !cached, &B.pA, &B.blkA, &B.ablk0, &shA,
                          &ncA, cached ? &shA : nullptr));
  SCUC_TRY(tune_partition(B, true, rpts, B.col0_h, B.nnz0_h, autotune && !cached, &B.pT, &B.blkT, &B.tblk0, &shT,
                          &ncT, cached ? &shT : nullptr));
  if (autotune && !cached) remember_shapes(key, shA, shT);
  const double tune_ms = std::chrono::duration<double, std::milli>(clk::now() - tt0).count();
  if (autotune && !cached) launches += 4 * (int64_t)(ncA + ncT);
  int maxn = 1;
  for (int b = 0; b < nlp; b++) maxn = std::max(maxn, H[b]->n);
  B.epi_gx = std::max(1, std::min(64, (maxn + kBlock - 1) / kBlock));
  SCUC_TRY(B.alloc(&B.gsum, n));
  SCUC_TRY(B.alloc(&B.gsum32, n));
  SCUC_TRY(B.alloc(&B.partP, 4 * (size_t)B.epi_gx * nlp));
  SCUC_TRY(B.alloc(&B.partD, 2 * (size_t)B.pA.nblk));
  SCUC_TRY(B.alloc(&B.partRA, 3 * (size_t)B.pA.nblk));
  SCUC_TRY(B.alloc(&B.partRT, (size_t)B.pT.nblk));

  // 4. per-LP control blocks, Halpern weights of the first period, logs
  const int ce = p.check_every;
  B.coef_stride = 2 * ce;
  B.log_cap = 4096;
  SCUC_TRY(B.alloc(&B.ctrl, nlp));
  SCUC_TRY(B.alloc(&B.coef, (size_t)nlp * B.coef_stride));
  SCUC_TRY(B.alloc(&B.log, (size_t)nlp * B.log_cap));
  SCUC_CUDA(cudaMallocHost((void**)&B.ctrl_h, 2 * (size_t)nlp * sizeof(Ctrl)));
  std::vector<double> coef_h((size_t)nlp * B.coef_stride);
  for (int b = 0; b < nlp; b++) {
    Ctrl& c = C[b];
    c.tol = p.tol;
    c.sigma = p.sigma0;
    c.lambda = lam[b];
    c.restart_suff = p.restart_suff;
    c.restart_nec = p.restart_nec;
    c.restart_long = p.restart_long;
    c.restart_ref = p.restart_ref;
    c.restart_metric = p.restart_metric;
    c.sigma_update = p.sigma_update;
    c.algo = SCUC_ALGO_HPR;
    c.infeas_tol = 0.0;
    c.s_step = 1.0 / (lam[b] * p.sigma0);
    c.polish_factor = p.polish_factor;
    c.max_iter = ((p.max_iter + ce - 1) / ce) * ce;
    c.check_every = ce;
    c.polish_stall = p.polish_stall;
    c.polish_floor = p.polish_floor;
    c.log_cap = B.log_cap;
    c.precision = p.precision;
    c.k = 0; c.t = 0; c.iters_fp32 = 0;
    c.rho0 = 0; c.rho_prev = 0; c.best_kkt = INFINITY;
    c.first_check = 1; c.done = 0; c.status = -1; c.restart_pending = 0;
    c.reject_kkt = 0.0;
    c.restarts = 0; c.nlog = 0; c.fp64_phase = mixed ? 0 : 1; c.stall = 0;
    for (int j = 0; j < ce; j++) {
      coef_h[(size_t)b * B.coef_stride + 2 * j] = 1.0 / (double)(j + 2);
      coef_h[(size_t)b * B.coef_stride + 2 * j + 1] = (double)(j + 1) / (double)(j + 2);
    }
  }
  SCUC_CUDA(cudaMemcpyAsync(B.coef, coef_h.data(), coef_h.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  int maxdim = 1;
  for (int b = 0; b < nlp; b++) maxdim = std::max(maxdim, std::max(H[b]->m, H[b]->n));
  const int ga = std::max(1, std::min(64, (maxdim + kBlock - 1) / kBlock));
  const DevLP L = B.dev();
  SCUC_CUDA(cudaStreamSynchronize(s));
  const auto t1 = clk::now();

  // 5. iterations: one graph launch (the device loops until every LP has
  // stopped), or one period at a time from the host, two in flight
  const int64_t nper = C[0].max_iter / ce;
  const bool use_graph = p.use_graph != 0;
  const int64_t per_launch = period_launches(B, ce);
  int64_t periods = 0;
  int timed_out = 0;
  for (int b = 0; b < nlp; b++) {
    C[b].t_start_ns = 0;
    C[b].time_limit_ns = (p.time_limit_s > 0.0 && p.time_limit_s < 1e9) ? (uint64_t)(p.time_limit_s * 1e9) : 0;
  }
  SCUC_CUDA(cudaMemcpyAsync(B.ctrl, C.data(), nlp * sizeof(Ctrl), cudaMemcpyHostToDevice, s));
  k_init_iterates<<<dim3(ga, nlp), kBlock, 0, s>>>(L, nullptr, nullptr);
  launches++;
  SCUC_CUDA(cudaGetLastError());
  if (use_graph) {
    SCUC_TRY(build_batch_graph(B, ce, ga));
    SCUC_CUDA(cudaGraphLaunch(B.graph, s));
    SCUC_CUDA(cudaStreamSynchronize(s));
    SCUC_CUDA(cudaMemcpyAsync(C.data(), B.ctrl, nlp * sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaStreamSynchronize(s));
    int64_t tmax = 0;
    for (int b = 0; b < nlp; b++) tmax = std::max<int64_t>(tmax, C[b].t);
    periods = (tmax + ce - 1) / ce;
    launches += periods * (per_launch + 1);
  } else {
    int64_t launched = 0, seen = 0;
    while (seen < nper) {
      while (launched < nper && launched - seen < 2) {
        SCUC_TRY(launch_batch_period(B, s, ce, ga));
        launches += per_launch;
        SCUC_CUDA(cudaMemcpyAsync(B.ctrl_h + (size_t)(launched & 1) * nlp, B.ctrl, nlp * sizeof(Ctrl),
                                  cudaMemcpyDeviceToHost, s));
        SCUC_CUDA(cudaEventRecord(B.ev_slot[launched & 1], s));
        launched++;
      }
      SCUC_CUDA(cudaEventSynchronize(B.ev_slot[seen & 1]));
      const Ctrl* hc = B.ctrl_h + (size_t)(seen & 1) * nlp;
      seen++;
      periods++;
      bool all = true;
      for (int b = 0; b < nlp && all; b++) all = hc[b].done != 0;
      if (all) break;
      if (std::chrono::duration<double>(clk::now() - t0).count() > p.time_limit_s) {
        timed_out = 1;
        break;
      }
    }
    SCUC_CUDA(cudaStreamSynchronize(s));
    SCUC_CUDA(cudaMemcpyAsync(C.data(), B.ctrl, nlp * sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaStreamSynchronize(s));
  }
  const auto t2 = clk::now();

  // 6. unscaled outputs, logs, per-LP information
  k_finalize<<<dim3(ga, nlp), kBlock, 0, s>>>(L, B.xo, B.yo, B.zo);
  launches++;
  SCUC_CUDA(cudaGetLastError());
  const cudaMemcpyKind kind = p.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int b = 0; b < nlp; b++) {
    Handle& h = *H[b];
    const int r0 = B.row0_h[b], c0 = B.col0_h[b];
    if (xo && xo[b] && h.n) SCUC_CUDA(cudaMemcpyAsync(xo[b], B.xo + c0, h.n * sizeof(double), kind, s));
    if (zo && zo[b] && h.n) SCUC_CUDA(cudaMemcpyAsync(zo[b], B.zo + c0, h.n * sizeof(double), kind, s));
    if (yo && yo[b] && h.m) SCUC_CUDA(cudaMemcpyAsync(yo[b], B.yo + r0, h.m * sizeof(double), kind, s));
    SCUC_TRY(h.ensure_log(B.log_cap));
    const int nl = std::min(C[b].nlog, B.log_cap);
    if (nl)
      SCUC_CUDA(cudaMemcpyAsync(h.log_d, B.log + (size_t)b * B.log_cap, nl * sizeof(scuc_check_log),
                                cudaMemcpyDeviceToDevice, s));
    h.last_nlog = nl;
  }
  SCUC_CUDA(cudaStreamSynchronize(s));
  const auto t3 = clk::now();
  const double setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  const double solve_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
  for (int b = 0; b < nlp; b++) {
    scuc_solve_info& in = infos[b];
    memset(&in, 0, sizeof(in));
    const Ctrl& c = C[b];
    in.status = timed_out && !c.done ? SCUC_ST_TIME_LIMIT : (c.status < 0 ? SCUC_ST_ITER_LIMIT : c.status);
    in.restarts = c.restarts;
    in.iters = c.t;
    in.iters_fp32 = c.iters_fp32;
    in.power_iters = piters[b];
    in.nlog = std::min(c.nlog, B.log_cap);
    in.kkt = c.kkt; in.rp = c.rp; in.rd = c.rd; in.gap = c.gap;
    in.pobj = c.pobj; in.dobj = c.dobj;
    in.lambda = c.lambda; in.sigma = c.sigma; in.beta = c.beta; in.gamma = c.gamma;
    in.setup_ms = setup_ms;
    in.solve_ms = solve_ms;
    in.launches = launches;
  }
  if (bi) {
    bi->ept_A = shA.ept;
    bi->run_A = shA.min_run;
    bi->ept_T = shT.ept;
    bi->run_T = shT.min_run;
    bi->candidates = cached ? 0 : ncA + ncT;
    bi->tune_cached = cached ? 1 : 0;
    bi->scale_ms = std::chrono::duration<double, std::milli>(ts1 - t0).count();
    bi->setup_ms = setup_ms;
    bi->tune_ms = tune_ms;
    bi->solve_ms = solve_ms;
    bi->total_ms = std::chrono::duration<double, std::milli>(t3 - t0).count();
    bi->launches = launches;
    bi->periods = periods;
    bi->blocks_A = B.pA.nblk;
    bi->blocks_T = B.pT.nblk;
  }
  for (int b = 0; b < nlp; b++) SCUC_TRY(H[b]->leave());
  return SCUC_OK;
}

}  // namespace scuc
