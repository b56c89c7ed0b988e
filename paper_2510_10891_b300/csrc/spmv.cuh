// CSR SpMV core with a per-row epilogue hook (fused into the HPR steps).
//
// One CTA of kBlock threads per entry of a host-built partition; each entry
// is one of three block types, chosen from the row lengths:
//  * kLongRowBlock   (type 3): one row with more than kGroupRowMax nonzeros;
//    the whole block streams it and reduces with a fixed tree;
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
    const VT acc = block_sum(group_dot(col, val, x, ldg(rp + r), ldg(rp + r + 1), tid, kBlock));
    if (tid == 0) epi.row(r, acc);
    return;
  }
  if (d.x == kGroupListBlock) {
    const int gsz = d.w;  // 4, 8, 16 or 32 threads per row
    const int g = tid / gsz, li = tid - g * gsz;
    const bool act = g < d.z;
    const int r = act ? part.list[d.y + g] : 0;
    VT acc = act ? group_dot(col, val, x, ldg(rp + r), ldg(rp + r + 1), li, gsz) : VT(0);
    for (int off = gsz >> 1; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, gsz);
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
      for (int e = a + li; e < z; e += gsz) acc = fma_t(s_val[e], ldg(x + s_col[e]), acc);
    }
    for (int off = gsz >> 1; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, gsz);
    if (r < r1 && li == 0) epi.row(r, acc);
  }
}

}  // namespace scuc
