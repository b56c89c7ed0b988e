// CSR SpMV core with a per-row epilogue hook (fused into the HPR steps).
//
// One CTA of kBlock threads per entry of a host-built partition; each entry
// is one of four block types, chosen from the row lengths:
//  * kLongRowBlock   (type 3): one row with more than kWarpRowMax nonzeros; the
//    whole block streams it (4 independent accumulators per thread) and
//    reduces with a fixed tree;
//  * kWarpRowsBlock  (type 2): up to 8 rows of kShortMax+1..kWarpRowMax nonzeros
//    from a row list, one warp per row (4 accumulators per lane);
//  * kShortListBlock (type 1): up to 64 rows of <= kShortMax nonzeros from a row
//    list, 4 threads per row;
//  * kStagedBlock    (type 0): a contiguous run of short rows whose val/col slice
//    (<= kNnzCap entries) is staged in shared memory with coalesced loads,
//    then reduced by groups of gsz threads.
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

// Sum of val[e] * x[col[e]] for e = a, a + step, ... < z, four independent
// accumulators combined in a fixed order.
template <typename VT>
__device__ __forceinline__ VT strided_dot(const int* __restrict__ col, const VT* __restrict__ val,
                                          const VT* __restrict__ x, int a, int z, int step) {
  VT s0 = VT(0), s1 = VT(0), s2 = VT(0), s3 = VT(0);
  int e = a;
  for (; e + 3 * step < z; e += 4 * step) {
    const int c0 = ldcs(col + e), c1 = ldcs(col + e + step), c2 = ldcs(col + e + 2 * step),
              c3 = ldcs(col + e + 3 * step);
    const VT v0 = ldcs(val + e), v1 = ldcs(val + e + step), v2 = ldcs(val + e + 2 * step),
             v3 = ldcs(val + e + 3 * step);
    s0 = fma(v0, ldg(x + c0), s0);
    s1 = fma(v1, ldg(x + c1), s1);
    s2 = fma(v2, ldg(x + c2), s2);
    s3 = fma(v3, ldg(x + c3), s3);
  }
  for (; e < z; e += step) s0 = fma(ldcs(val + e), ldg(x + ldcs(col + e)), s0);
  return (s0 + s1) + (s2 + s3);
}

// Runs the SpMV of one partition entry; calls epi.row(r, acc) once per row,
// from a single thread.  smem must hold kNnzCap * (sizeof(VT) + 4) bytes.
template <typename VT, class Epi>
__device__ __forceinline__ void spmv_block(const int* __restrict__ rp, const int* __restrict__ col,
                                           const VT* __restrict__ val, const VT* __restrict__ x,
                                           const Partition& part, unsigned char* smem, Epi& epi) {
  const int4 d = part.desc[blockIdx.x];  // {type, first, count, gsz}
  const int tid = threadIdx.x;
  if (d.x == kLongRowBlock) {
    const int r = part.list[d.y];
    const VT acc = block_sum(strided_dot(col, val, x, ldg(rp + r) + tid, ldg(rp + r + 1), kBlock));
    if (tid == 0) epi.row(r, acc);
    return;
  }
  if (d.x == kWarpRowsBlock) {
    const int w = tid >> 5, lane = tid & 31;
    if (w < d.z) {
      const int r = part.list[d.y + w];
      VT acc = strided_dot(col, val, x, ldg(rp + r) + lane, ldg(rp + r + 1), 32);
      acc = warp_sum(acc);
      if (lane == 0) epi.row(r, acc);
    }
    return;
  }
  if (d.x == kShortListBlock) {
    const int g = tid >> 2, li = tid & 3;
    const bool act = g < d.z;
    const int r = act ? part.list[d.y + g] : 0;
    VT acc = VT(0);
    if (act) {
      const int z = ldg(rp + r + 1);
      for (int e = ldg(rp + r) + li; e < z; e += 4) acc = fma(ldcs(val + e), ldg(x + ldcs(col + e)), acc);
    }
    acc += __shfl_down_sync(0xffffffffu, acc, 2, 4);
    acc += __shfl_down_sync(0xffffffffu, acc, 1, 4);
    if (act && li == 0) epi.row(r, acc);
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
      for (int e = a + li; e < z; e += gsz) acc = fma(s_val[e], ldg(x + s_col[e]), acc);
    }
    for (int off = gsz >> 1; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, gsz);
    if (r < r1 && li == 0) epi.row(r, acc);
  }
}

}  // namespace scuc
