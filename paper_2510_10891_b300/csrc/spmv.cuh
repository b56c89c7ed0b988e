// CSR SpMV core with a per-row epilogue hook (fused into the HPR steps).
//
// Layout: one CTA of kBlock threads per row block of a host-built partition.
//  * multi-row block (gsz >= 1): the block's contiguous slice of val/col is
//    staged in shared memory with coalesced loads, then groups of gsz
//    threads reduce one row each (gsz = 1: thread per row, sequential in
//    column order); partial sums of a group are combined with a fixed
//    shuffle tree, so results are deterministic run to run;
//  * long-row block (gsz == 0): the whole block streams the row's
//    val/col directly (fully coalesced) and reduces with a fixed tree.
// Exactly one fused multiply-add per nonzero: on B300 the FP64 pipe is the
// second roofline of an FP64 SpMV, so products are never formed separately.
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

// Runs the SpMV of one row block; calls epi.row(r, acc) once per row, from a
// single thread.  smem must hold kNnzCap * (sizeof(VT) + 4) bytes.
template <typename VT, class Epi>
__device__ __forceinline__ void spmv_block(const int* __restrict__ rp, const int* __restrict__ col,
                                           const VT* __restrict__ val, const VT* __restrict__ x,
                                           const Partition& part, unsigned char* smem, Epi& epi) {
  const int b = blockIdx.x;
  const int r0 = part.row[b], r1 = part.row[b + 1];
  const int gsz = part.gsz[b];
  const int tid = threadIdx.x;
  if (gsz == 0) {
    const int e0 = rp[r0], e1 = rp[r0 + 1];
    VT acc = VT(0);
    int e = e0 + tid;
    // two independent accumulators keep two loads in flight per thread
    VT acc2 = VT(0);
    for (; e + kBlock < e1; e += 2 * kBlock) {
      acc = fma(ldg(val + e), ldg(x + ldg(col + e)), acc);
      acc2 = fma(ldg(val + e + kBlock), ldg(x + ldg(col + e + kBlock)), acc2);
    }
    if (e < e1) acc = fma(ldg(val + e), ldg(x + ldg(col + e)), acc);
    acc = block_sum(acc + acc2);
    if (tid == 0) epi.row(r0, acc);
    return;
  }
  VT* s_val = reinterpret_cast<VT*>(smem);
  int* s_col = reinterpret_cast<int*>(smem + kNnzCap * sizeof(VT));
  const int e0 = rp[r0], e1 = rp[r1];
  for (int e = e0 + tid; e < e1; e += kBlock) {
    s_val[e - e0] = ldg(val + e);
    s_col[e - e0] = ldg(col + e);
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
