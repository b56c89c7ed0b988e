// CSR SpMV core with a per-row epilogue hook (fused into the HPR steps).
//
// Long rows (more than kSellMaxLen nonzeros in the partitions of one LP:
// the dense PTDF, N-1, balance and reserve rows) are cut into chunks of
// kChunk entries; a
// chunk launch (k_chunk_sums and friends) gives every chunk one warp that
// streams it with coalesced lane-strided loads (the whole chunk in flight
// for FP32 values, eight entries per lane at a time for FP64) and stores the
// chunk sum (FP32 values: from the chunk stream, 16-byte value and 8-byte
// offset loads, columns as 16-bit offsets from one of two bases per chunk
// where the chunk's columns allow).  The main launch gives every long row one
// thread that adds its chunk sums in chunk order and runs the epilogue; its
// other blocks are
//  * list blocks: kBlock/gsz rows of similar length, gsz = 32, 16, 8 or 4
//    threads per row, each row's entry range read from one 16-byte record;
//  * staged blocks: a contiguous run of short rows whose val/col slice
//    (<= kNnzCap entries) is staged in shared memory with coalesced loads,
//    then reduced by groups of gsz threads.
// A block first loads what it needs to know about its rows (spmv_plan: one
// record per row or per run, no value type), so that a kernel can issue
// those loads together with its own control loads before it picks the
// precision of the products (spmv_run).  Every thread that will run an
// epilogue row calls epi.load(row) first, so the epilogue's operands are
// fetched while the row is being summed; the row sums go through shared
// memory so the epilogue runs one row per thread with full warps.
// The chain of dependent loads before the first product is short (record ->
// matrix entries -> gathered vector) because blocks are short-lived and
// thousands of them run back to back.
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

// Deterministic block reduction of Q per-thread values into out[q * stride
// + slot].
template <int Q>
__device__ __forceinline__ void block_store_slot(const double (&v)[Q], double* out, int stride, int slot) {
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
      out[q * stride + slot] = s;
    }
  }
}

// partials of a main SpMV launch: block b writes slot part.slot[b] (or b)
template <int Q>
__device__ __forceinline__ void block_store(const double (&v)[Q], double* out, const Partition& part) {
  block_store_slot<Q>(v, out, part.nblk, part.slot ? part.slot[blockIdx.x] : (int)blockIdx.x);
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
// increasing order, mostly a few apart).  Entries go in batches of U per
// thread whose loads are all issued before the first product; entry e + u*nl
// of a batch goes to accumulator u mod NA, and the NA accumulators are
// combined in a fixed tree.  PRED: the last partial batch is one predicated
// batch (a row of 100 entries over 16 threads is then a single batch);
// otherwise its entries are added one dependent load at a time into the
// first accumulator.  Measured on the 13k-bus LP: list rows U = 12, NA = 2
// with predication for FP32 values (U at least the 12 entries per thread of
// the default partition, so most rows take one batch; U = 16 costs
// occupancy); for FP64 values, which are bound by B300's FP64 pipe (2 DFMA
// per clock per SM) rather than by loads in flight, U = 4 without
// predication and a single accumulator (no combining adds).
template <typename VT, int U, int NA, bool PRED>
__device__ __forceinline__ VT batched_dot(const int* __restrict__ col, const VT* __restrict__ val,
                                          const VT* __restrict__ x, int e, int z, int nl) {
  VT s[NA];
#pragma unroll
  for (int q = 0; q < NA; q++) s[q] = VT(0);
  for (; e + (U - 1) * nl < z; e += U * nl) {
    int c[U];
    VT v[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      c[u] = ldcs(col + e + u * nl);
      v[u] = ldcs(val + e + u * nl);
    }
#pragma unroll
    for (int u = 0; u < U; u++) s[u % NA] = fma_t(v[u], ldg(x + c[u]), s[u % NA]);
  }
  if (!PRED) {
    for (; e < z; e += nl) s[0] = fma_t(ldcs(val + e), ldg(x + ldcs(col + e)), s[0]);
  } else if (e < z) {
    int c[U];
    VT v[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int q = e + u * nl;
      c[u] = q < z ? ldcs(col + q) : -1;
      v[u] = q < z ? ldcs(val + q) : VT(0);
    }
#pragma unroll
    for (int u = 0; u < U; u++)
      if (c[u] >= 0) s[u % NA] = fma_t(v[u], ldg(x + c[u]), s[u % NA]);
  }
#pragma unroll
  for (int w = NA / 2; w > 0; w >>= 1)
#pragma unroll
    for (int q = 0; q < w; q++) s[q] += s[q + w];
  return s[0];
}

// The group size nl a compile-time constant (FP32 values: the loads of a
// batch address their entries with immediate offsets from one pointer).
template <typename VT, int nl>
__device__ __forceinline__ VT group_dot(const int* __restrict__ col, const VT* __restrict__ val,
                                        const VT* __restrict__ x, int a, int z, int li) {
  return batched_dot<VT, sizeof(VT) == 4 ? 12 : 4, 2, sizeof(VT) == 4>(col, val, x, a + li, z, nl);
}

// The same with the group size known only at run time (measured faster for
// FP64 values on the 13k-bus A^T; the compile-time form is faster for FP32).
template <typename VT>
__device__ __forceinline__ VT group_dot_rt(const int* __restrict__ col, const VT* __restrict__ val,
                                           const VT* __restrict__ x, int a, int z, int li, int nl) {
  return batched_dot<VT, sizeof(VT) == 4 ? 8 : 4, sizeof(VT) == 4 ? 8 : 1, sizeof(VT) == 4>(col, val, x,
                                                                                               a + li, z, nl);
}

// FP32 chunk sums (one warp per chunk of at most kChunk = 512 entries).
// Lane l takes entries i = 128u + 4l + k (groups u = 0..3 in order, k =
// 0..3), entry k into accumulator k & 1, then adds its two accumulators;
// the warp sum follows.  Entries past the chunk's end count as value 0 at
// the chunk's last column.  From the chunk stream (Partition::cst) a lane
// reads each group's 4 values with one 16-byte load and their 4 column
// offsets with one 8-byte load (6 bytes per entry instead of 8 on a product
// bound by HBM), all issued at once from the chunk's index alone (the
// record's place is fixed), the chunk's bases (crec) alongside; entry i's
// column is (i < split ? base0 : base1) + offset (TWO: the chunk has a
// second cluster; otherwise every entry uses base0, a warp-uniform choice
// per chunk).  chunk32_sum: the same order on the CSR arrays with 32-bit
// columns (chunks that need them, or no stream), so both give the same sum
// bit for bit.
__device__ __forceinline__ void chunk16_load(const Partition& part, int w, int lane, float4 (&v)[kChunk / 128],
                                             uint2 (&o)[kChunk / 128]) {
  const float4* __restrict__ vp = reinterpret_cast<const float4*>(part.cst + (size_t)w * kChunkRec16);
  const uint2* __restrict__ op = reinterpret_cast<const uint2*>(vp + kChunk / 4);
#pragma unroll
  for (int u = 0; u < kChunk / 128; u++) {
    v[u] = ldcs(vp + 32 * u + lane);
    o[u] = ldcs(op + 32 * u + lane);
  }
}

template <bool TWO>
__device__ __forceinline__ float chunk16_sum(int4 rec, const float4 (&v)[kChunk / 128],
                                             const uint2 (&o)[kChunk / 128], const float* __restrict__ x, int lane) {
  const int split = rec.z & 0xffff;
  const float* __restrict__ x0 = x + rec.x;
  const float* __restrict__ x1 = x + rec.y;
  float s[2] = {0.f, 0.f};
#pragma unroll
  for (int u = 0; u < kChunk / 128; u++) {
    const int i = 128 * u + 4 * lane;
    const float vv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
    const unsigned cc[4] = {o[u].x & 0xffffu, o[u].x >> 16, o[u].y & 0xffffu, o[u].y >> 16};
#pragma unroll
    for (int k = 0; k < 4; k++) s[k & 1] = fma_t(vv[k], ldg((TWO && i + k >= split ? x1 : x0) + cc[k]), s[k & 1]);
  }
  return s[0] + s[1];
}

__device__ __forceinline__ float chunk32_sum(const int* __restrict__ col, const float* __restrict__ val,
                                             const float* __restrict__ x, int2 c, int lane) {
  float s[2] = {0.f, 0.f};
#pragma unroll
  for (int u = 0; u < kChunk / 128; u++)
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int e = c.x + 128 * u + 4 * lane + k;
      const bool in = e < c.y;
      s[k & 1] = fma_t(in ? ldcs(val + e) : 0.0f, ldg(x + ldcs(col + (in ? e : c.y - 1))), s[k & 1]);
    }
  return s[0] + s[1];
}

// One warp per chunk of a long row (chunk launch): chunk w = blockIdx.x *
// (kBlock / 32) + warp; for FP32 values chunk16_sum / chunk32_sum (the whole
// chunk, 16 entries per lane, in flight at once), for FP64 lane-strided
// batches of 8 into one accumulator (FP64-pipe bound: eight accumulators
// cost seven combining adds per 16 products, 20% of the dual step); then a
// fixed warp tree; the sum goes to part.cpart[w] in FP64.
// cb: the block's index among the chunk blocks (blockIdx.x unless a launch
// interleaves them with other work); WPB: warps per block of the launch.
template <typename VT, int WPB = kBlock / 32>
__device__ __forceinline__ void chunk_warp(const int* __restrict__ col, const VT* __restrict__ val,
                                           const VT* __restrict__ x, const Partition& part,
                                           int cb = -1) {
  const int w = (cb < 0 ? (int)blockIdx.x : cb) * WPB + (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= part.nchunk) return;
  VT s;
  if constexpr (sizeof(VT) == 4) {
    // the chunk stream once it is filled, unless the chunk needs 32-bit columns
    if (part.cst) {
      float4 v[kChunk / 128];
      uint2 o[kChunk / 128];
      chunk16_load(part, w, lane, v, o);
      const int4 rec = part.crec[w];
      if (rec.x < 0) s = chunk32_sum(col, val, x, part.chunks[w], lane);
      else if ((rec.z & 0xffff) >= (rec.z >> 16)) s = chunk16_sum<false>(rec, v, o, x, lane);
      else s = chunk16_sum<true>(rec, v, o, x, lane);
    } else {
      s = chunk32_sum(col, val, x, part.chunks[w], lane);
    }
  } else {
    const int2 c = part.chunks[w];
    s = batched_dot<VT, 8, 1, false>(col, val, x, c.x + lane, c.y, 32);
  }
  s = warp_sum(s);
  if (lane == 0) part.cpart[w] = (double)s;
}

// Sum of long row li's chunk sums, in chunk order: loaded eight at a time
// so a row of many chunks (a 21,000-entry row has 41) waits for one batch,
// not one load per chunk; the adds keep their order (the same result).
// One thread per row: B300's FP64 pipe makes a sum that every lane of a
// warp repeats cost 32 times as much.
__device__ __forceinline__ double chunk_total(const Partition& part, int li) {
  int c = part.chunk_ptr[li];
  const int ce = part.chunk_ptr[li + 1];
  double s = 0.0;
  for (; c + 8 <= ce; c += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; u++) v[u] = part.cpart[c + u];
#pragma unroll
    for (int u = 0; u < 8; u++) s += v[u];
  }
  for (; c < ce; c++) s += part.cpart[c];
  return s;
}

// The same sum in predicated batches of sixteen (three batches for 41
// chunks), for kernels with registers to spare (the long-row launch).
__device__ __forceinline__ double chunk_total16(const Partition& part, int li) {
  int c = part.chunk_ptr[li];
  const int ce = part.chunk_ptr[li + 1];
  double s = 0.0;
  for (; c < ce; c += 16) {
    double v[16];
#pragma unroll
    for (int u = 0; u < 16; u++) v[u] = c + u < ce ? part.cpart[c + u] : 0.0;
#pragma unroll
    for (int u = 0; u < 16; u++)
      if (c + u < ce) s += v[u];
  }
  return s;
}

// What a block of the main launch needs to know about its rows, loaded
// before the value type is chosen.
struct BlockPlan {
  int kind;   // 0 list, 1 staged, 2 long rows
  int gsz;    // threads per row (list, staged)
  int cnt;    // rows of the block (list: rows incl. padding; staged: rows)
  int4 rec;   // list: this thread's group's row {row, first, end}; staged: the run
  int er;     // row whose epilogue this thread runs, -1: none
  int li;     // long rows: index into long_rows
};

// WITH_ER: also load the epilogue row of each thread (not needed when the
// group leaders store their sums directly).
// b: the block's index among the partition's main blocks (blockIdx.x
// unless a launch interleaves them with other work).
template <bool WITH_ER = true>
__device__ __forceinline__ BlockPlan spmv_plan(const Partition& part, int b) {
  BlockPlan bp;
  const int tid = threadIdx.x;
  const int nlist = part.cls_blk[4];
  bp.er = -1;
  bp.li = -1;
  if (b < nlist) {
    int k = 0;
    while (k < 3 && b >= part.cls_blk[k + 1]) k++;
    bp.kind = 0;
    bp.gsz = 32 >> k;
    const int per = kBlock / bp.gsz;
    const int i0 = part.cls_row[k] + (b - part.cls_blk[k]) * per;
    bp.cnt = min(per, part.cls_row[k + 1] - i0);
    const int g = tid / bp.gsz;
    bp.rec = g < bp.cnt ? part.listx[i0 + g] : make_int4(-1, 0, 0, 0);
    if (WITH_ER && tid < bp.cnt) bp.er = part.listx[i0 + tid].x;
  } else if (b < nlist + part.nstaged) {
    bp.kind = 1;
    bp.rec = part.desc[b - nlist];
    bp.cnt = bp.rec.w >> 8;
    bp.gsz = bp.rec.w & 255;
    if (tid < bp.cnt) bp.er = bp.rec.x + tid;
  } else {
    bp.kind = 2;
    bp.gsz = 1;
    bp.cnt = 0;
    bp.rec = make_int4(0, 0, 0, 0);
    const int i = (b - nlist - part.nstaged) * kBlock + tid;
    if (i < part.nlong) {
      bp.li = i;
      bp.er = part.long_rows[i];
    }
  }
  return bp;
}

template <bool WITH_ER = true>
__device__ __forceinline__ BlockPlan spmv_plan(const Partition& part) {
  return spmv_plan<WITH_ER>(part, (int)blockIdx.x);
}

// Runs the SpMV of the block planned in bp; calls epi.row(r, acc) once per
// row, from the thread with bp.er == r (which called epi.load(r) before).
// smem must hold part.smem bytes (dynamic).
// DIRECT: the group leader calls epi.row itself (no shared-memory pass, no
// barrier) -- for epilogues that only store the sum.
template <typename VT, class Epi, bool DIRECT = false>
__device__ __forceinline__ void spmv_run(const BlockPlan& bp, const int* __restrict__ rp,
                                         const int* __restrict__ col, const VT* __restrict__ val,
                                         const VT* __restrict__ x, const Partition& part, unsigned char* smem,
                                         Epi& epi) {
  const int tid = threadIdx.x;
  if (bp.kind == 2) {
    if (bp.li >= 0) epi.row(bp.er, (VT)chunk_total(part, bp.li));
    return;
  }
  VT* s_sum = reinterpret_cast<VT*>(smem + kNnzCap * 12);
  if (bp.kind == 0) {
    const int gsz = bp.gsz;
    const int g = tid / gsz, li = tid - g * gsz;
    VT acc = VT(0);
    if (bp.rec.x >= 0) {
      if (sizeof(VT) == 8) {
        acc = group_dot_rt<VT>(col, val, x, bp.rec.y, bp.rec.z, li, gsz);
      } else {
        switch (gsz) {
          case 32: acc = group_dot<VT, 32>(col, val, x, bp.rec.y, bp.rec.z, li); break;
          case 16: acc = group_dot<VT, 16>(col, val, x, bp.rec.y, bp.rec.z, li); break;
          case 8: acc = group_dot<VT, 8>(col, val, x, bp.rec.y, bp.rec.z, li); break;
          default: acc = group_dot<VT, 4>(col, val, x, bp.rec.y, bp.rec.z, li); break;
        }
      }
    }
    for (int off = gsz >> 1; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, gsz);
    if (DIRECT) {
      if (li == 0 && bp.rec.x >= 0) epi.row(bp.rec.x, acc);
      return;
    }
    if (li == 0 && g < bp.cnt) s_sum[g] = acc;
    __syncthreads();
    if (bp.er >= 0) epi.row(bp.er, s_sum[tid]);
    return;
  }
  // staged contiguous run of short rows: rows [r0, r0 + nr), entries [e0, e1)
  VT* s_val = reinterpret_cast<VT*>(smem);
  int* s_col = reinterpret_cast<int*>(smem + kNnzCap * sizeof(VT));
  int* s_rp = reinterpret_cast<int*>(smem + kNnzCap * 12 + kBlock * 8);
  const int r0 = bp.rec.x, e0 = bp.rec.y, e1 = bp.rec.z, nr = bp.cnt, gsz = bp.gsz;
  if (tid < nr) s_rp[tid] = ldg(rp + r0 + tid);
  if (tid == 0) s_rp[nr] = e1;
  for (int e = e0 + tid; e < e1; e += kBlock) {
    s_val[e - e0] = ldcs(val + e);
    s_col[e - e0] = ldcs(col + e);
  }
  __syncthreads();
  const int gi = tid / gsz, li = tid - gi * gsz, ng = kBlock / gsz;
  for (int base = 0; base < nr; base += ng) {
    const int q = base + gi;
    VT acc = VT(0);
    if (q < nr) {
      const int a = s_rp[q] - e0, z = s_rp[q + 1] - e0;
      for (int e = a + li; e < z; e += gsz) acc = fma_t(s_val[e], ldg(x + s_col[e]), acc);
    }
    for (int off = gsz >> 1; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, gsz);
    if (gsz == 1 || DIRECT) {  // epilogue directly from the row's leader
      if (q < nr && li == 0) epi.row(r0 + q, acc);
    } else if (q < nr && li == 0) {
      s_sum[q] = acc;
    }
  }
  if (gsz > 1 && !DIRECT) {
    __syncthreads();
    if (bp.er >= 0) epi.row(bp.er, s_sum[tid]);
  }
}

// Plan, epilogue loads and run in one call (for kernels with no control loads).
template <typename VT, class Epi>
__device__ __forceinline__ void spmv_block(const int* __restrict__ rp, const int* __restrict__ col,
                                           const VT* __restrict__ val, const VT* __restrict__ x,
                                           const Partition& part, unsigned char* smem, Epi& epi) {
  const BlockPlan bp = spmv_plan<true>(part);
  if (bp.er >= 0) epi.load(bp.er);
  spmv_run<VT>(bp, rp, col, val, x, part, smem, epi);
}

// Chunk launch of a partition with long rows: grid part.nchunkblk.
template <typename VT>
__global__ void __launch_bounds__(kBlock) k_chunk_sums(const int* __restrict__ col, const VT* __restrict__ val,
                                                       const VT* __restrict__ x, Partition part) {
  chunk_warp<VT>(col, val, x, part);
}

}  // namespace scuc
