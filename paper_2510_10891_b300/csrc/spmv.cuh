// CSR SpMV core with a per-row epilogue hook (fused into the HPR steps).
//
// Rows with more than kGroupRowMax nonzeros are streamed by persistent CTAs
// (blocks [0, nstream)): one thread issues 1-D bulk copies (cp.async.bulk,
// completion on an mbarrier) of kTile-entry tiles of the row's indices and
// values into a kStages-deep shared-memory ring, so the matrix stream never
// waits on the gathers; all threads then gather and accumulate from shared
// memory and reduce with a fixed tree at each row's end.  Every other block
// runs one entry of a host-built partition, one of two types:
//  * kGroupListBlock (type 1): kBlock/gsz rows from a row list, gsz = 4, 8,
//    16 or 32 threads per row chosen from the row length;
//  * kStagedBlock    (type 0): a contiguous run of short rows whose val/col
//    slice (<= kNnzCap entries) is staged in shared memory with coalesced
//    loads, then reduced by groups of gsz threads.
// Long and list rows are read lane-strided (consecutive lanes, consecutive
// entries), four entries in flight per thread.
// All reductions have a fixed order, so results are deterministic run to
// run.  Exactly one fused multiply-add per nonzero (FP64 issues at 2 DFMA per
// clock per SM on B300, so products are never formed separately).  Matrix
// values and indices are read with evict-first loads: they are streamed once
// per launch, while the gathered vector should stay in L2.
#pragma once
#include "common.cuh"

namespace scuc {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// Deterministic block sum; the result is valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum(T v) {
  __shared__ T s_part[kBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();  // s_part may still be read by a previous call
  if (lane == 0) s_part[warp] = v;
  __syncthreads();
  T r = T(0);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < kBlock / 32; w++) r += s_part[w];
  }
  return r;
}

// Deterministic block reduction of Q per-thread values; thread 0 writes
// out[q * stride + blockIdx.x].
template <int Q>
__device__ __forceinline__ void block_store(const double (&v)[Q], double* out, int stride) {
  __shared__ double s_q[Q][kBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < Q; q++) {
    double w = warp_sum(v[q]);
    if (lane == 0) s_q[q][warp] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < Q; q++) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kBlock / 32; w++) s += s_q[q][w];
      out[q * stride + blockIdx.x] = s;
    }
  }
}

template <typename T>
__device__ __forceinline__ T ldg(const T* p) {
  return __ldg(p);
}

// streamed once per launch: evict-first
template <typename T>
__device__ __forceinline__ T ldcs(const T* p) {
  return __ldcs(p);
}

// fused multiply-add in the value type (explicit, so nothing is promoted)
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

// Partial sum of val[e] * x[col[e]] for e = a + li, a + li + nl, ... < z:
// consecutive lanes take consecutive entries, so one warp-wide gather touches
// neighbouring columns (rows of these matrices list their columns in
// increasing order, mostly a few apart); four independent accumulators,
// combined in a fixed order.
template <typename VT>
__device__ __forceinline__ VT group_dot(const int* __restrict__ col, const VT* __restrict__ val,
                                        const VT* __restrict__ x, int a, int z, int li, int nl) {
  VT s0 = VT(0), s1 = VT(0), s2 = VT(0), s3 = VT(0);
  int e = a + li;
  for (; e + 3 * nl < z; e += 4 * nl) {
    const int c0 = ldcs(col + e), c1 = ldcs(col + e + nl), c2 = ldcs(col + e + 2 * nl),
              c3 = ldcs(col + e + 3 * nl);
    const VT v0 = ldcs(val + e), v1 = ldcs(val + e + nl), v2 = ldcs(val + e + 2 * nl),
             v3 = ldcs(val + e + 3 * nl);
    s0 = fma_t(v0, ldg(x + c0), s0);
    s1 = fma_t(v1, ldg(x + c1), s1);
    s2 = fma_t(v2, ldg(x + c2), s2);
    s3 = fma_t(v3, ldg(x + c3), s3);
  }
  for (; e < z; e += nl) s0 = fma_t(ldcs(val + e), ldg(x + ldcs(col + e)), s0);
  return (s0 + s1) + (s2 + s3);
}

// ---- bulk-copy (TMA) ring for long rows -----------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 1-D bulk copy global -> shared, completion counted on bar (16-byte aligned
// addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Waits for the given phase of bar within a clock budget; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitBudgetCycles) return false;
  return true;
}

// tile sequence of a streaming CTA: rows long_rows[c], c = blockIdx.x +
// k * nstream, each cut into kTile-entry tiles
struct TileIt {
  int c, e, rend, row;
  __device__ void start(const Partition& P, const int* rp) {
    c = blockIdx.x;
    if (c < P.nlong) {
      row = P.long_rows[c];
      e = rp[row];
      rend = rp[row + 1];
    }
  }
  __device__ bool valid(const Partition& P) const { return c < P.nlong; }
  __device__ void next(const Partition& P, const int* rp) {
    e += kTile;
    if (e >= rend) {
      c += P.nstream;
      if (c < P.nlong) {
        row = P.long_rows[c];
        e = rp[row];
        rend = rp[row + 1];
      }
    }
  }
};

// Issues the bulk copies of the tile at `it` into ring stage `st`.
template <typename VT>
__device__ __forceinline__ void issue_tile(const TileIt& it, const int* col, const VT* val, unsigned char* ring,
                                           uint64_t* bars, int st) {
  const int e1 = min(it.e + kTile, it.rend);
  const int ea = it.e & ~3, eb = (e1 + 3) & ~3;  // 16-byte aligned span (arrays are padded)
  const uint32_t nb_col = (uint32_t)(eb - ea) * 4u, nb_val = (uint32_t)(eb - ea) * (uint32_t)sizeof(VT);
  unsigned char* stage = ring + st * kStageBytes;
  mbar_arrive_expect_tx(bars + st, nb_col + nb_val);
  bulk_g2s(stage, col + ea, nb_col, bars + st);
  bulk_g2s(stage + (kTile + kTileSlack) * 4, val + ea, nb_val, bars + st);
}

// Persistent streaming of the long rows: tid 0 keeps kStages tiles in flight;
// all threads read each tile from shared memory (thread t: entries t,
// t + kBlock, ...), gather x and accumulate; at a row's last tile a fixed
// block reduction feeds epi.row.
template <typename VT, class Epi>
__device__ void stream_long_rows(const int* __restrict__ rp, const int* __restrict__ col,
                                 const VT* __restrict__ val, const VT* __restrict__ x, const Partition& P,
                                 unsigned char* smem, Epi& epi) {
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  unsigned char* ring = smem + 128;
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < kStages; s++) mbar_init(bars + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  __syncthreads();
  TileIt prod, cons;
  prod.start(P, rp);
  cons.start(P, rp);
  int issued = 0;
  if (tid == 0)
    for (; issued < kStages && prod.valid(P); issued++, prod.next(P, rp)) issue_tile<VT>(prod, col, val, ring, bars, issued);
  VT a0 = VT(0), a1 = VT(0);
  for (int k = 0; cons.valid(P); k++) {
    const int st = k % kStages;
    if (!mbar_wait_bounded(bars + st, (uint32_t)((k / kStages) & 1))) s_fail = 1;
    __syncthreads();
    if (s_fail) break;
    const unsigned char* stage = ring + st * kStageBytes;
    const int ea = cons.e & ~3;
    const int* s_col = reinterpret_cast<const int*>(stage);  // entry e at [e - ea]
    const VT* s_val = reinterpret_cast<const VT*>(stage + (kTile + kTileSlack) * 4);
    const int e1 = min(cons.e + kTile, cons.rend);
    // this thread's (at most kPerThread) entries of the tile: indices and
    // values from shared memory first, then all gathers, then the FMAs
    constexpr int kPerThread = (kTile + kBlock - 1) / kBlock;
    int cc[kPerThread];
    VT vv[kPerThread], xx[kPerThread];
#pragma unroll
    for (int q = 0; q < kPerThread; q++) {
      const int e = cons.e + tid + q * kBlock;
      cc[q] = e < e1 ? s_col[e - ea] : -1;
      vv[q] = e < e1 ? s_val[e - ea] : VT(0);
    }
#pragma unroll
    for (int q = 0; q < kPerThread; q++) xx[q] = cc[q] >= 0 ? ldg(x + cc[q]) : VT(0);
#pragma unroll
    for (int q = 0; q < kPerThread; q++) {
      if (q & 1) a1 = fma_t(vv[q], xx[q], a1);
      else a0 = fma_t(vv[q], xx[q], a0);
    }
    const bool last = e1 >= cons.rend;
    const int row = cons.row;
    __syncthreads();  // stage st fully read
    if (tid == 0 && prod.valid(P)) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_tile<VT>(prod, col, val, ring, bars, st);
      prod.next(P, rp);
      issued++;
    }
    if (last) {
      const VT acc = block_sum(a0 + a1);
      if (tid == 0) epi.row(row, acc);
      a0 = VT(0);
      a1 = VT(0);
    }
    cons.next(P, rp);
  }
  if (s_fail) {
    // a wait ran out: record it and let copies still in flight land (bounded)
    if (tid == 0) {
      atomicOr(P.err, 1);
      for (int s = 0; s < kStages; s++) mbar_wait_bounded(bars + s, 0u), mbar_wait_bounded(bars + s, 1u);
    }
    __syncthreads();
  }
}

// Runs the SpMV of one partition entry; calls epi.row(r, acc) once per row,
// from a single thread.  smem must hold part.smem bytes (dynamic).
template <typename VT, class Epi>
__device__ __forceinline__ void spmv_block(const int* __restrict__ rp, const int* __restrict__ col,
                                           const VT* __restrict__ val, const VT* __restrict__ x,
                                           const Partition& part, unsigned char* smem, Epi& epi) {
  if ((int)blockIdx.x < part.nstream) {
    stream_long_rows<VT>(rp, col, val, x, part, smem, epi);
    return;
  }
  const int4 d = part.desc[blockIdx.x - part.nstream];  // {type, first, count, gsz}
  const int tid = threadIdx.x;
  // row sums of the block (behind the staging buffer), so that the epilogue
  // runs one row per thread with full warps (a warp instruction costs the
  // FP64 pipe the same however few of its lanes are active)
  // Launches that also stream long rows are limited by shared memory to a few
  // CTAs per SM; there the extra barrier costs more than it saves, so rows go
  // straight to the epilogue from their group leader.
  const bool smem_epi = part.nstream == 0;
  VT* s_sum = reinterpret_cast<VT*>(smem + kNnzCap * 12);
  int* s_row = reinterpret_cast<int*>(smem + kNnzCap * 12 + kBlock * 8);
  if (d.x == kGroupListBlock) {
    const int gsz = d.w;  // 4, 8, 16 or 32 threads per row
    const int g = tid / gsz, li = tid - g * gsz;
    const bool act = g < d.z;
    const int r = act ? part.list[d.y + g] : 0;
    VT acc = act ? group_dot(col, val, x, ldg(rp + r), ldg(rp + r + 1), li, gsz) : VT(0);
    for (int off = gsz >> 1; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, gsz);
    if (!smem_epi) {
      if (act && li == 0) epi.row(r, acc);
      return;
    }
    if (act && li == 0) {
      s_sum[g] = acc;
      s_row[g] = r;
    }
    __syncthreads();
    if (tid < d.z) epi.row(s_row[tid], s_sum[tid]);
    return;
  }
  // staged contiguous run of short rows
  VT* s_val = reinterpret_cast<VT*>(smem);
  int* s_col = reinterpret_cast<int*>(smem + kNnzCap * sizeof(VT));
  const int r0 = d.y, r1 = d.y + d.z, gsz = d.w;
  const int e0 = ldg(rp + r0), e1 = ldg(rp + r1);
  for (int e = e0 + tid; e < e1; e += kBlock) {
    s_val[e - e0] = ldcs(val + e);
    s_col[e - e0] = ldcs(col + e);
  }
  __syncthreads();
  const int gi = tid / gsz, li = tid - gi * gsz, ng = kBlock / gsz;
  for (int base = r0; base < r1; base += ng) {
    const int r = base + gi;
    VT acc = VT(0);
    if (r < r1) {
      const int a = ldg(rp + r) - e0, z = ldg(rp + r + 1) - e0;
      for (int e = a + li; e < z; e += gsz) acc = fma_t(s_val[e], ldg(x + s_col[e]), acc);
    }
    for (int off = gsz >> 1; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, gsz);
    if (gsz == 1 || !smem_epi) {  // thread per row, or direct epilogue
      if (r < r1 && li == 0) epi.row(r, acc);
    } else if (r < r1 && li == 0) {
      s_sum[r - r0] = acc;
    }
  }
  if (gsz > 1 && smem_epi) {
    __syncthreads();
    if (tid < r1 - r0) epi.row(r0 + tid, s_sum[tid]);
  }
}

}  // namespace scuc
