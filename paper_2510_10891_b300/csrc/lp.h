// Internal declarations of the SCUC LP library (host side).
#pragma once
#include <memory>
#include <utility>
#include <vector>

#include "common.cuh"

namespace scuc {

struct DevLP;      // device view of a handle (lp_kernels.cuh)
struct Validator;  // input checks of scuc_lp_create, run while the arrays are copied (lp.cu)

// A^T of a matrix built elsewhere (Handle::init_device adopts the arrays,
// and the two host row-pointer arrays: they are moved from)
struct DevTranspose {
  int *rpt, *colt, *permt;
  double* valt;
  std::vector<int>* rp_h;   // row pointers of A (m + 1)
  std::vector<int>* rpt_h;  // row pointers of A^T (n + 1)
};

// allocator whose resize leaves new elements default-initialised (for a
// trivial type: unwritten), for buffers the planner writes in full
template <typename T>
struct NoInitAlloc : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <typename U>
  NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <typename U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <typename U, typename... Args>
  void construct(U* p, Args&&... args) {
    ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
  }
};

// host plan of a Partition
struct PartPlan {
  std::vector<int4, NoInitAlloc<int4>> listx;  // every list row is written by plan_partition
  std::vector<int4> desc;
  std::vector<int> long_rows, chunk_ptr, slot;
  std::vector<int2> chunks;
  int cls_blk[5] = {0, 0, 0, 0, 0};
  int cls_row[5] = {0, 0, 0, 0, 0};
  void clear() {  // empty, capacity kept
    listx.clear(); desc.clear(); long_rows.clear(); chunk_ptr.clear(); slot.clear(); chunks.clear();
    for (int k = 0; k < 5; k++) cls_blk[k] = cls_row[k] = 0;
  }
};
int build_partition(const std::vector<int>& rp, int m, Partition* P, int long_min = kGroupRowMax);
// sliced ELL structure of a CSR matrix with row pointers rp (the FP32 value
// arrays are chosen and allocated by Handle::sell_values, the values filled
// on the device by k_sell_fill); freed with the handle's allocations
// (rows longer than max_len are left out: their sums come from elsewhere)
int build_sell(const std::vector<int>& rp, int m, int max_len, Sell* S, std::vector<void*>* allocs);
void plan_partition(const std::vector<int>& rp, int m, const PartShape& shape, bool allow_long, PartPlan* plan,
                    int long_min = kGroupRowMax);
int upload_partition(const PartPlan& plan, Partition* P);
void free_partition(Partition* P);
int exclusive_scan(const int* in, int n, int* out, cudaStream_t s);
int dev_alloc_bytes(void** p, size_t bytes);  // from the device's pool (lp.cu)
void dev_free(void* p);                       // back to the pool; the caller has drained its users

struct Handle {
  int32_t m = 0, n = 0;
  int64_t nnz = 0;
  int device = 0;
  cudaStream_t user = nullptr, work = nullptr;
  cudaEvent_t ev_user = nullptr, ev_work = nullptr, ev_slot[2] = {nullptr, nullptr};
  std::vector<void*> allocs;
  // matrix
  int *rp = nullptr, *col = nullptr, *rpt = nullptr, *colt = nullptr, *permt = nullptr;
  double *val = nullptr, *valt = nullptr, *vs = nullptr, *vst = nullptr;
  float *vs32 = nullptr, *vst32 = nullptr;
  Partition pA, pT;
  Sell sT;  // sliced ELL copy of A^T's rows of <= kSellMaxLen nonzeros (primal step)
  Sell sA;  // the same of A's rows when A has chunked rows (dual step of plain iterations)
  std::vector<int> rpt_plan;  // row pointers of A^T until sT is built (at the first solve)
  std::vector<int> rp_plan;   // row pointers of A until sA is built (A with chunked rows)
  bool sell_planned = false;
  // problem data (unscaled and scaled)
  double *c = nullptr, *xl = nullptr, *xu = nullptr, *lo = nullptr, *hi = nullptr;
  double *Dr = nullptr, *Dc = nullptr, *cs = nullptr, *xls = nullptr, *xus = nullptr,
         *los = nullptr, *his = nullptr;
  // iterates and scratch
  double *x = nullptr, *x0 = nullptr, *xt = nullptr, *xbar = nullptr, *zbar = nullptr;
  double *y = nullptr, *y0 = nullptr, *ybar = nullptr;
  float *xt32 = nullptr, *y32 = nullptr;
  double* dychk = nullptr;
  double* dxchk = nullptr;  // x_bar - x of a check (infeasibility detection)
  double *qv = nullptr, *uv = nullptr, *wv = nullptr;
  double *partP = nullptr, *partD = nullptr, *partRA = nullptr, *partRT = nullptr;
  double* gsum = nullptr;  // A^T y of the primal step (FP64 phases)
  float* gsum32 = nullptr;  // ... (FP32 phases)
  int epi_gx = 1;          // blocks of the primal epilogue
  Ctrl* ctrl = nullptr;
  Ctrl* ctrl_h = nullptr;
  PowerCtrl* pctrl = nullptr;
  scuc_check_log* log_d = nullptr;
  int log_cap = 0, last_nlog = 0;
  cudaGraphExec_t graph_exec = nullptr;
  // check_every, FP32 values, log, coef, initial phase, algorithm, detection, layout
  const void* graph_key[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaStream_t aux = nullptr;  // capture stream of the graph's conditional bodies
  double* coef = nullptr;
  int64_t nlaunch = 0, graph_nodes = 0;  // kernels launched by this handle; nodes of the period graph
  int coef_cap = 0;
  std::vector<double> coef_h;
  std::vector<cudaEvent_t> prof_ev;

  ~Handle();
  template <typename T>
  int alloc(T** p, size_t count);
  int init(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
           const double* val, const double* c, const double* xl, const double* xu,
           const double* lo, const double* hi, cudaStream_t user, Validator* check = nullptr);
  int begin(int32_t m, int32_t n, int64_t nnz, cudaStream_t user);
  int init_device(int32_t m, int32_t n, int64_t nnz, int* d_rp, int* d_col, double* d_val, double* d_c,
                  double* d_xl, double* d_xu, double* d_lo, double* d_hi, cudaStream_t user,
                  const DevTranspose* t = nullptr);
  int setup_device(std::vector<int>& rp32);
  int build_transpose(std::vector<int>* rpt_h);
  int setup_solver(std::vector<int>& rp32, std::vector<int>& rpt_h);
  // FP32 value form of a sliced ELL copy built by build_sell (compressed
  // when asked and every row allows it, else the 32-bit form)
  int sell_values(Sell* S, const int* rp_d, const int* col_d, bool compress);
  // FP32 chunk stream of a partition (at the first FP32 set-up)
  int chunk_stream(Partition* P, const int* col_d, int which);
  bool index16 = true;                     // FP32 products may read 16-bit offsets (scuc_lp_set_index16)
  unsigned long long* n16_d = nullptr;     // [2] entries of A's / A^T's chunks using offsets
  unsigned long long n16_h[2] = {0, 0};
  int enter();
  int leave();
  DevLP dev() const;
  int setup_scaling(int use_scaling, bool need_f32);
  int power_method(const scuc_solve_params& p, double* lam, int* iters);
  int power_start(const scuc_solve_params& p);
  int power_round(const scuc_solve_params& p);
  int power_poll(const scuc_solve_params& p, bool* done, double* lam, int* iters);
  PowerCtrl* pctrl_host = nullptr;  // pinned copy of the power method's state
  cudaEvent_t ev_power = nullptr;
  bool power_f32 = false;
  bool power_sell = false;  // FP32 power iterations run A^T on the sliced copy
  int power_rounds = 0;
  int ensure_log(int cap);
  template <int PREC>
  int launch_iterations(cudaStream_t s, int check_every, bool profile);
  int launch_checks(cudaStream_t s, int check_every);
  int64_t period_kernels(int check_every) const;
  int algo = SCUC_ALGO_HPR;  // of the current solve (kernels launched by the checks)
  bool use_sell = false;     // the current solve's primal products run on sT
  bool split_steps = false;  // the current solve keeps product and update apart on plain iterations
  bool use_sell_dual = false;  // the current solve's plain dual steps run k_dual_fused
  bool detect = false;       // infeasibility detection in the current solve
  int launch_period(int check_every, bool profile, bool fp64);
  int build_solve_graph(int check_every, int phase64);
  // keep_scaling: the caller has changed nothing since this handle's last
  // solve, so its scaled data (set up for the same use_scaling and
  // precision) is reused instead of recomputed (the warm-start path's
  // solves after its cold reference period)
  int solve(const scuc_solve_params& p, const double* x0, const double* y0, double* xo,
            double* yo, double* zo, scuc_solve_info* info, double reject_kkt = 0.0,
            bool keep_scaling = false);
  int scaled_for = -1;  // use_scaling + 256 * (FP32 copies) of the scaled data; -1: none
  int* pt_flag = nullptr;  // index checks of scuc_ws_assemble / scuc_ws_targets
  // rows [0, m) then columns [m, m + n): short ones (<= 32 entries) first,
  // each group in index order (built at the first fixing call)
  int* fix_lists = nullptr;
  int fix_short_rows = 0, fix_short_cols = 0;
  int build_fix_lists();
  int matvec(int transpose, const double* in, double* out);
  int kkt_noalloc(const double* x, const double* y, const double* z, double* out);
  int fix_and_propagate(const scuc_map& map, const uint8_t* is_int, const double* x, const scuc_fix_params& p,
                        int8_t* fix_out, Handle** reduced, int32_t* col_map, int32_t* row_map, scuc_fix_info* info);
  int row_violations(const double* x, int on_device, double tol, int32_t* rows_out, int32_t cap, int32_t* count_out,
                     double* worst_out);
  int add_rows(const Handle& pool, const int32_t* rows, int32_t count, Handle** out);
  int get_bounds(double* xl, double* xu);
  int set_bounds(const double* xl, const double* xu, int on_device);
  int export_lp(int64_t* row_ptr, int32_t* col, double* val, double* c, double* xl, double* xu, double* lo,
                double* hi);
};

int create_handle(Handle** out, int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                  const int32_t* col, const double* val, const double* c, const double* xl,
                  const double* xu, const double* lo, const double* hi, void* stream);

// scuc_lp_solve_batch (batch.cu)
int solve_batch(Handle* const* H, int nlp, const scuc_solve_params& p, double* const* xo, double* const* yo,
                double* const* zo, scuc_solve_info* infos, scuc_batch_info* bi);

}  // namespace scuc

// C-ABI handle (include/scuc_lp.h)
struct scuc_lp {
  scuc::Handle* h;
};
