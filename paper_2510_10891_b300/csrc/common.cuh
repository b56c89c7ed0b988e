// Shared definitions of the sm_103a SCUC LP library (device + host).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "scuc_lp.h"

namespace scuc {

void set_error(const char* fmt, ...);

#define SCUC_CUDA(expr)                                                                  \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess) {                                                             \
      ::scuc::set_error("%s: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, __LINE__); \
      return _e == cudaErrorMemoryAllocation ? SCUC_E_OOM : SCUC_E_CUDA;                 \
    }                                                                                    \
  } while (0)

#define SCUC_TRY(expr)              \
  do {                              \
    int _r = (expr);                \
    if (_r != SCUC_OK) return _r;   \
  } while (0)

constexpr int kBlock = 256;        // threads per SpMV block
constexpr int kNnzCap = 2048;      // nonzeros staged in shared memory per staged block
constexpr int kMaxRows = 256;      // rows per staged block
constexpr int kShortMax = 32;        // short rows: <= this many nonzeros
constexpr int kGroupRowMax = 4096;   // list rows up to this many; longer rows get a block
constexpr int kDecideThreads = 1024;

// block types of a partition entry
constexpr int kStagedBlock = 0, kGroupListBlock = 1;

// threads per row of a list row: about ept entries per thread, 4..32
inline int group_size_for(int len, int ept = 16) {
  int g = 4;
  while (g < 32 && g * ept < len) g *= 2;
  return g;
}

// tunable shape of a partition (plan_partition)
struct PartShape {
  int ept = 16;      // target entries per thread of list rows
  int min_run = 32;  // shortest run of short rows that is staged in shared memory
};

// streamed long rows: tiles of kTile entries, kStages-deep shared-memory ring
constexpr int kTile = 960;
constexpr int kStages = 4;
constexpr int kTileSlack = 8;                                   // alignment slack (entries)
constexpr int kStageBytes = (kTile + kTileSlack) * 12;          // int index + FP64 value
constexpr int kStreamSmem = 128 + kStages * kStageBytes;        // mbarriers + ring
// the SpMV kernels keep static shared memory small so that the ring fits
// under the 48 KB a launch may take without a function attribute
static_assert(kStreamSmem + 1024 <= 48 * 1024, "streaming ring must fit the default shared memory");
constexpr int kStagedSmem = kNnzCap * 12 + kBlock * 12;  // staging + row sums/ids
constexpr long long kWaitBudgetCycles = 4000000000LL;           // ~2 s at 2 GHz

// Partition of a CSR matrix for the SpMV kernels.  Blocks [0, nstream) are
// persistent CTAs that stream the long rows (long_rows[c], c = blockIdx,
// blockIdx + nstream, ...) through shared memory with bulk copies; block
// nstream + b runs desc[b] = {type, first, count, gsz}: staged blocks cover
// rows [first, first + count) with gsz threads per row, list blocks cover
// rows list[first .. first + count).  nblk = nstream + number of desc
// entries (grid size and number of partial-sum slots).
struct Partition {
  int nblk = 0;
  int nstream = 0;
  int nlong = 0;
  int smem = kStagedSmem;        // dynamic shared memory of a launch
  int4* desc = nullptr;
  int* list = nullptr;
  int* long_rows = nullptr;
  int* err = nullptr;            // set to 1 when a bounded wait runs out
};

// Device-resident solver state.  Parameters are written by the host before a
// solve; the state is advanced only by the decide kernel.
struct Ctrl {
  double tol, sigma, lambda, beta, gamma, bnorm, cnorm;
  double restart_suff, restart_nec, restart_long, polish_factor;
  int64_t max_iter;
  int32_t check_every, polish_stall, log_cap, precision, restart_ref, restart_metric;
  int64_t k, t, iters_fp32;
  double rho0, rho_prev, best_kkt, s_step;
  int32_t sigma_update, pad1;
  int32_t first_check, done, status, restart_pending;
  int32_t restarts, nlog, fp64_phase, stall;
  double kkt, rp, rd, gap, pobj, dobj;
  double reject_kkt;  // > 0: stop with SCUC_ST_FALLBACK_COLD if the first check has kkt >= this
};

struct PowerCtrl {
  double lam, lam_prev, nw, tol;
  int32_t it, max_iter, done, pad;
};

}  // namespace scuc
