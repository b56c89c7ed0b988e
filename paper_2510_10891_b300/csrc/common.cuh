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
constexpr int kMaxRows = 256;      // rows per staged block (<= kBlock: one epilogue row per thread)
constexpr int kShortMax = 32;        // short rows: <= this many nonzeros
constexpr int kGroupRowMax = 4096;   // list rows up to this many; longer rows get a block
constexpr int kDecideThreads = 1024;
// resident blocks per SM the dual-step kernel asks for (register cap 40:
// measured faster than 64 registers at half the occupancy)
constexpr int kDualMinBlocks = 6;
static_assert(kMaxRows <= 256, "a staged block's rows map to its threads");


// threads per row of a list row: about ept entries per thread, 4..32
inline int group_size_for(int len, int ept = 16) {
  int g = 4;
  while (g < 32 && g * ept < len) g *= 2;
  return g;
}

// tunable shape of a partition (plan_partition)
// Defaults measured on the 13k-bus LP (FP32 A^T product: 0.319 ms at 12
// entries per thread, 0.331 at 16, 0.441 at 24; 6-10 within 1 %).
struct PartShape {
  int ept = 12;      // target entries per thread of list rows
  int min_run = 32;  // shortest run of short rows that is staged in shared memory
};

constexpr int kChunk = 512;             // entries per chunk of a long row (one warp each)
constexpr int kSpan16 = 65535;          // widest column span a 16-bit offset covers
// staging (values + indices), row sums, row pointers of a staged run
constexpr int kStagedSmem = kNnzCap * 12 + kBlock * 8 + (kMaxRows + 1) * 4;

// Partition of a CSR matrix for the SpMV kernels (spmv.cuh).  Long rows
// are cut into chunks; a chunk launch (nchunkblk blocks, one chunk per warp)
// stores the chunk sums in cpart before the main launch.  The main launch
// has nblk blocks:
//  * list blocks [0, cls_blk[4]): class k = 0..3 (blocks [cls_blk[k],
//    cls_blk[k+1])) reads rows with 32 >> k threads per row, kBlock / (32 >>
//    k) consecutive entries of listx[cls_row[k] .. cls_row[k+1]) per block;
//  * staged blocks [cls_blk[4], cls_blk[4] + nstaged): desc[b - cls_blk[4]];
//  * long-row blocks: one thread per long row adds its chunk sums in order.
// Block b writes its partial sums to slot[b] (nullptr: slot b).
struct Partition {
  int nblk = 0;
  int cls_blk[5] = {0, 0, 0, 0, 0};
  int cls_row[5] = {0, 0, 0, 0, 0};
  int nstaged = 0;
  int nlong = 0;
  int nchunk = 0;
  int nchunkblk = 0;
  int64_t nchunk_ent = 0;        // entries in chunks
  int smem = kStagedSmem;        // dynamic shared memory of a main launch
  int4* listx = nullptr;         // list rows {row, first entry, end entry, 0}; row -1 pads a block
  int4* desc = nullptr;          // staged runs {first row, first entry, end entry, (rows << 8) | gsz}
  int2* chunks = nullptr;        // [nchunk] entry range [x, y) of each chunk, long row by long row
  int* long_rows = nullptr;      // [nlong]
  int* chunk_ptr = nullptr;      // [nlong + 1] first chunk of each long row
  double* cpart = nullptr;       // [nchunk] chunk sums
  int* slot = nullptr;           // [nblk] partial-sum slot of each block, or nullptr
  // FP32 chunk stream (allocated at the first FP32 set-up; nullptr until
  // then): chunk w's entries as one 3,072-byte record at cst + w *
  // kChunkRec16: its kChunk FP32 values, then kChunk 16-bit column offsets
  // (a shorter chunk padded with value 0 and its last entry's offset), so a
  // warp can load a chunk's entries before it knows anything else about the
  // chunk.  A chunk's columns (sorted) fall into at most two clusters of
  // span <= kSpan16: crec[w] = {base0, base1, (len << 16) | split, 0},
  // chunk-local entry i has column (i < split ? base0 : base1) + offset[i];
  // base0 = -1 marks a chunk that needs more clusters (its FP32 products
  // read the CSR arrays with 32-bit columns).
  uint4* cst = nullptr;          // [nchunk * kChunkRec16]
  int4* crec = nullptr;          // [nchunk]
};

// 16-byte units of a chunk record: kChunk values (4 bytes) + offsets (2 bytes)
constexpr int kChunkRec16 = kChunk * 6 / 16;


// Sliced ELL copy of a CSR matrix (used for A^T in the primal step): rows
// go in slices of 32, one row per lane; entry k of the row in lane r of
// slice s sits at (sptr[s] + k) * 32 + r, so a warp reads one slice step
// with one coalesced request.  Rows are sorted by length within windows of
// kSellWindow consecutive rows (neighbouring columns of the SCUC LP share
// most of their rows, so the lanes of a slice gather nearby vector
// entries); slices run longest first.  A row shorter than its slice is
// padded with its last column and a zero value.
constexpr int kSellWindow = 4096;
// rows longer than this are cut into kChunk-entry chunks (one warp each) in
// the partitions of a single LP; the sliced ELL copies hold the others (a
// lane walks its row alone, so longer rows would serialise their slice)
constexpr int kSellMaxLen = 512;
struct Sell {
  int nslice = 0;
  int64_t nent = 0;       // entries incl. padding (= sptr[nslice] * 32)
  int* sptr = nullptr;    // [nslice + 1] first step of each slice
  int* rows = nullptr;    // [nslice * 32] row of each lane, -1: none
  int2* cv32 = nullptr;   // [nent] {column, FP32 value bits} (not compressed)
  int* col = nullptr;     // [nent] column (FP64 values)
  double* v64 = nullptr;  // [nent] FP64 value
  // Compressed FP32 form (compressed = 1; then cv32 is not allocated): the
  // columns of a row fall into at most two clusters, each spanning at most
  // 65,535, so an entry is its FP32 value and a 16-bit offset from its
  // cluster's first column.  lrec[lane of slice] = {row, base0, base1,
  // kjump}: steps k < kjump are offsets from base0, the others from base1.
  // Steps go in pairs: pair p of lane r of slice s sits at (pptr[s] + p) *
  // 32 + r in v2 (the two FP32 values) and o2 (the two offsets, step 2p in
  // the low half), so a warp reads one pair of steps with two coalesced
  // requests (256 + 128 bytes).
  int compressed = 0;
  int* pptr = nullptr;        // [nslice + 1] first pair of each slice
  int4* lrec = nullptr;       // [nslice * 32]
  float2* v2 = nullptr;       // [pptr[nslice] * 32]
  unsigned* o2 = nullptr;     // [pptr[nslice] * 32]
  int64_t npair = 0;          // pptr[nslice]
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
  int32_t sigma_update, algo;  // algo: SCUC_ALGO_HPR or SCUC_ALGO_PDHG_AVG
  int32_t first_check, done, status, restart_pending;
  int32_t restarts, nlog, fp64_phase, stall;
  double kkt, rp, rd, gap, pobj, dobj;
  double reject_kkt;  // > 0: stop with SCUC_ST_FALLBACK_COLD if the first check has kkt >= this
  uint64_t t_start_ns;     // device clock at the start of the iterations
  uint64_t time_limit_ns;  // > 0: stop with SCUC_ST_TIME_LIMIT after this long (checked at checks)
  double infeas_tol;       // > 0: infeasibility detection at checks (relative certificate violation)
  double polish_floor;     // MIXED: FP64 matvecs from kkt <= max(polish_factor * tol, polish_floor)
};

struct PowerCtrl {
  double lam, lam_prev, nw, tol;
  int32_t it, max_iter, done, pad;
};

}  // namespace scuc
