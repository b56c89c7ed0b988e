// Warm-start network (scuc_ws_* in include/scuc_ws.h): a multilayer
// perceptron with hand-written forward, backward and Adam kernels.
//
// GEMMs run on the tensor cores with BF16 operands and FP32 accumulation.
// The hidden layers' forward products H W (K and N up to 256: all but a
// few per cent of the network's flops) run on the fifth-generation tensor
// cores: operands brought into shared memory by TMA, tcgen05.mma issued by
// one thread with the accumulator in tensor memory, and an epilogue that
// reads it back with tcgen05.ld and adds the bias, the ReLU and the BF16
// copy for the next layer.  The other products (the first layer's 12
// inputs, the 3 outputs, the weight gradient H^T dZ split over the batch
// and the input gradient dZ W^T with FP32 dZ) use one mma.sync kernel whose
// operands are converted to BF16 while they are staged in shared memory.
// Master weights, biases and Adam moments are FP32.  Every reduction (batch
// loss, bias gradient, split-K partial products) has a fixed order, so
// training is deterministic.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda.h>  // CUtensorMap (the encoder is reached through the runtime)
#include <cuda_bf16.h>

#include "../../include/scuc_ws.h"
#include "common.cuh"

namespace scuc {
int dev_alloc_bytes(void** p, size_t bytes);
void dev_free(void* p);

namespace {

constexpr int kGemmThreads = 128;  // 4 warps, each 16 rows x 64 columns of the tile
constexpr int kTM = 64, kTN = 64, kTK = 16;
constexpr int kSplitMax = 16;      // split-K slices of the weight-gradient product
constexpr int kColParts = 32;      // row chunks of the bias-gradient sum
constexpr int kHeads = 3;

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// C[M x N] = sum_k A(i,k) B(k,j) over k in this slice's range.  A(i,k) =
// A[i*sa_i + k*sa_k], B(k,j) = B[k*sb_k + j*sb_j]; one stride of each operand
// is 1 and the loads walk that dimension, so they coalesce in either layout.
// blockIdx.z selects the K slice [z*kchunk, (z+1)*kchunk) and the output
// slice C + z*c_stride.  Zero padding covers ragged M, N and K.
template <typename TA, typename TB>
__global__ void __launch_bounds__(kGemmThreads) k_gemm(int M, int N, int K, int kchunk, const TA* __restrict__ A,
                                                       int64_t sa_i, int64_t sa_k, const TB* __restrict__ B,
                                                       int64_t sb_k, int64_t sb_j, float* __restrict__ C,
                                                       int64_t ldc, int64_t c_stride) {
  __shared__ __align__(16) __nv_bfloat16 sA[kTM][kTK + 8];  // [row][k], rows padded to 48 bytes
  __shared__ __align__(16) __nv_bfloat16 sB[kTN][kTK + 8];  // [col][k]
  const int i0 = blockIdx.y * kTM, j0 = blockIdx.x * kTN;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  C += (int64_t)blockIdx.z * c_stride;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gid = lane >> 2, tig = lane & 3;
  const bool a_kfast = sa_k == 1, b_jfast = sb_j == 1;
  float acc[8][4];
#pragma unroll
  for (int t = 0; t < 8; t++)
#pragma unroll
    for (int q = 0; q < 4; q++) acc[t][q] = 0.f;
  for (int k0 = kbeg; k0 < kend; k0 += kTK) {
#pragma unroll
    for (int e = 0; e < kTM * kTK / kGemmThreads; e++) {
      const int idx = tid + e * kGemmThreads;
      const int r = a_kfast ? idx / kTK : idx % kTM;
      const int k = a_kfast ? idx % kTK : idx / kTM;
      const int gi = i0 + r, gk = k0 + k;
      const float v = (gi < M && gk < kend) ? to_f(A[gi * sa_i + gk * sa_k]) : 0.f;
      sA[r][k] = __float2bfloat16_rn(v);
    }
#pragma unroll
    for (int e = 0; e < kTN * kTK / kGemmThreads; e++) {
      const int idx = tid + e * kGemmThreads;
      const int c = b_jfast ? idx % kTN : idx / kTK;
      const int k = b_jfast ? idx / kTN : idx % kTK;
      const int gj = j0 + c, gk = k0 + k;
      const float v = (gj < N && gk < kend) ? to_f(B[gk * sb_k + gj * sb_j]) : 0.f;
      sB[c][k] = __float2bfloat16_rn(v);
    }
    __syncthreads();
    // A fragment: rows gid and gid+8 of this warp's 16, k pairs 2*tig and 2*tig+8
    const int ra = warp * 16 + gid;
    uint32_t a[4];
    a[0] = *reinterpret_cast<const uint32_t*>(&sA[ra][2 * tig]);
    a[1] = *reinterpret_cast<const uint32_t*>(&sA[ra + 8][2 * tig]);
    a[2] = *reinterpret_cast<const uint32_t*>(&sA[ra][2 * tig + 8]);
    a[3] = *reinterpret_cast<const uint32_t*>(&sA[ra + 8][2 * tig + 8]);
#pragma unroll
    for (int t = 0; t < 8; t++) {
      // B fragment: column gid of the 8-wide tile t, k pairs 2*tig and 2*tig+8
      const int cb = t * 8 + gid;
      uint32_t b[2];
      b[0] = *reinterpret_cast<const uint32_t*>(&sB[cb][2 * tig]);
      b[1] = *reinterpret_cast<const uint32_t*>(&sB[cb][2 * tig + 8]);
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    __syncthreads();
  }
  // accumulator: rows gid / gid+8, columns 2*tig, 2*tig+1 of each 8-wide tile
#pragma unroll
  for (int t = 0; t < 8; t++) {
    const int r = i0 + warp * 16 + gid, c = j0 + t * 8 + 2 * tig;
    if (r < M) {
      if (c < N) C[(int64_t)r * ldc + c] = acc[t][0];
      if (c + 1 < N) C[(int64_t)r * ldc + c + 1] = acc[t][1];
    }
    if (r + 8 < M) {
      if (c < N) C[(int64_t)(r + 8) * ldc + c] = acc[t][2];
      if (c + 1 < N) C[(int64_t)(r + 8) * ldc + c + 1] = acc[t][3];
    }
  }
}

// ---------------------------------------------------------------------------
// Tensor-core GEMM on tcgen05: Z[rows x N] = act(H[rows x K] W[K x N] + b)
// for K a multiple of 64 up to 256 and N a multiple of 16 up to 256.  One
// CTA of 4 warps takes 128 rows.  Thread 0 loads the CTA's H rows and all of
// W^T (K-major, BF16) with TMA in 128-byte-swizzled chunks of 64 K values
// (one mbarrier counts the bytes), then issues K/16 tcgen05.mma of
// 128 x N x 16 into a TMEM accumulator of 128 lanes x N columns and commits
// them to a second mbarrier.  Each warp then reads its 32 lanes (rows) with
// tcgen05.ld and writes Z (FP32; null: not kept) and the BF16 copy.  Waits are bounded: a
// wait that runs out sets *err, waits once more for the copies in flight,
// skips the products and frees the TMEM.
// ---------------------------------------------------------------------------
constexpr int kTcM = 128, kTcThreads = 128, kTcKc = 64;
constexpr int kTcMaxK = 256, kTcMaxN = 256;
constexpr long long kTcSpin = 1LL << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// true once the phase with the given parity has completed; false after
// kTcSpin polls
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < kTcSpin; i++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in 128-byte
// swizzle: rows of 128 bytes (64 BF16), 8-row atoms of 1,024 bytes (the
// stride between atoms), leading offset unused in this mode.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__global__ void __launch_bounds__(kTcThreads, 1) k_gemm_tc(const __grid_constant__ CUtensorMap tmap_h,
                                                          const __grid_constant__ CUtensorMap tmap_w, int rows,
                                                          int N, int K, uint32_t tmem_cols,
                                                          const float* __restrict__ bias, int relu,
                                                          float* __restrict__ Z, __nv_bfloat16* __restrict__ Hb,
                                                          int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_tma, bar_mma;
  __shared__ uint32_t s_tmem;
  __shared__ int s_ok;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // swizzle atoms need 1,024-byte alignment
  const int nk = K / kTcKc;
  const uint32_t a_bytes = kTcM * 128u, b_bytes = (uint32_t)N * 128u;
  const uint32_t sa = base, sb = base + (uint32_t)nk * a_bytes;
  const int m0 = blockIdx.x * kTcM;
  const uint32_t btma = smem_u32(&bar_tma), bmma = smem_u32(&bar_mma);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    mbar_init(btma, 1);
    mbar_init(bmma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  if (threadIdx.x == 0) {
    int ok = 1;
    mbar_expect_tx(btma, (uint32_t)nk * (a_bytes + b_bytes));
    for (int kc = 0; kc < nk; kc++) {
      tma_load_2d(sa + (uint32_t)kc * a_bytes, &tmap_h, kc * kTcKc, m0, btma);
      tma_load_2d(sb + (uint32_t)kc * b_bytes, &tmap_w, kc * kTcKc, 0, btma);
    }
    if (!mbar_wait(btma, 0)) {
      ok = 0;
      atomicOr(err, 1);
      mbar_wait(btma, 0);  // once more for the copies in flight
    }
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t idesc = idesc_bf16(kTcM, N);
      for (int kc = 0; kc < nk; kc++)
        for (int ks = 0; ks < kTcKc / 16; ks++) {
          const uint64_t ad = umma_desc_sw128(sa + (uint32_t)kc * a_bytes + (uint32_t)ks * 32u);
          const uint64_t bd = umma_desc_sw128(sb + (uint32_t)kc * b_bytes + (uint32_t)ks * 32u);
          const uint32_t acc = (kc | ks) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bmma)
                   : "memory");
    }
    s_ok = ok;
  }
  __syncthreads();
  bool ok = s_ok != 0;
  if (ok && !mbar_wait(bmma, 0)) {
    atomicOr(err, 2);
    mbar_wait(bmma, 0);
    ok = false;
  }
  ok = __all_sync(0xffffffffu, ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < rows) {
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; q++) {
          float t = __uint_as_float(r[q]) + bias[c0 + q];
          v[q] = relu ? fmaxf(t, 0.f) : t;
        }
        if (Z) {
          float4* zp = reinterpret_cast<float4*>(Z + (int64_t)row * N + c0);
#pragma unroll
          for (int q = 0; q < 4; q++) zp[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        if (Hb) {
          __align__(16) __nv_bfloat16 h[16];
#pragma unroll
          for (int q = 0; q < 16; q++) h[q] = __float2bfloat16_rn(v[q]);
          uint4* hp = reinterpret_cast<uint4*>(Hb + (int64_t)row * N + c0);
          hp[0] = reinterpret_cast<const uint4*>(h)[0];
          hp[1] = reinterpret_cast<const uint4*>(h)[1];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// Wt[j][k] = W[k][j] (BF16, K x N -> N x K)
__global__ void k_transpose_bf16(int K, int N, const __nv_bfloat16* __restrict__ W, __nv_bfloat16* __restrict__ Wt) {
  const int64_t total = (int64_t)K * N, step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += step) {
    const int64_t j = e / K, k = e - j * K;
    Wt[e] = W[k * N + j];
  }
}

// out[e] = sum_{q < ns} parts[q*stride + e], slices in order
__global__ void k_sum_slices(int64_t count, int ns, int64_t stride, const float* __restrict__ parts,
                             float* __restrict__ out) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += step) {
    float s = 0.f;
    for (int q = 0; q < ns; q++) s += parts[q * stride + e];
    out[e] = s;
  }
}

// Xs[i, f] = (X[src_i, f] - mean_f) / scale_f with src_i = idx ? idx[i] : i;
// with Yb, also Yb[i, :] = Y[src_i, :]
__global__ void k_standardize(int rows, int F, const float* __restrict__ X, const int32_t* __restrict__ idx,
                              const float* __restrict__ mean, const float* __restrict__ scale,
                              float* __restrict__ Xs, const float* __restrict__ Y, float* __restrict__ Yb) {
  const int64_t total = (int64_t)rows * F, step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += step) {
    const int64_t i = e / F;
    const int f = (int)(e - i * F);
    const int64_t src = idx ? idx[i] : i;
    Xs[e] = (X[src * F + f] - mean[f]) / scale[f];
    if (Yb && f == 0)
      for (int c = 0; c < kHeads; c++) Yb[i * kHeads + c] = Y[src * kHeads + c];
  }
}

// Z = Z + b; hidden layers: Z = relu(Z) and a BF16 copy for the next product
__global__ void k_bias_act(int rows, int N, float* __restrict__ Z, const float* __restrict__ b, int relu,
                           __nv_bfloat16* __restrict__ Hb) {
  const int64_t total = (int64_t)rows * N, step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += step) {
    float v = Z[e] + b[e % N];
    if (relu) v = fmaxf(v, 0.f);
    Z[e] = v;
    if (Hb) Hb[e] = __float2bfloat16_rn(v);
  }
}

__device__ __forceinline__ float sigmoid(float z) { return 1.f / (1.f + expf(-z)); }

// out[i] = (sigmoid(o_0), sigmoid(o_1), o_2)
__global__ void k_heads(int rows, const float* __restrict__ O, float* __restrict__ out) {
  const int step = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += step) {
    const float* o = O + (int64_t)i * kHeads;
    float* q = out + (int64_t)i * kHeads;
    q[0] = sigmoid(o[0]);
    q[1] = sigmoid(o[1]);
    q[2] = o[2];
  }
}

constexpr int kLossThreads = 256;
constexpr int kLossBlocks = 148 * 4;

// Per-sample loss softplus(o0) - y0 o0 + w_d (sigmoid(o1) - y1)^2 +
// w_p (o2 - y2)^2, summed per block in a fixed order; dO = gradient of the
// batch mean.
__global__ void __launch_bounds__(kLossThreads) k_loss(int rows, const float* __restrict__ O,
                                                      const float* __restrict__ Y, float wd, float wp,
                                                      float* __restrict__ dO, double* __restrict__ part) {
  const float inv = 1.f / (float)rows;
  double l = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
    const float* o = O + (int64_t)i * kHeads;
    const float* y = Y + (int64_t)i * kHeads;
    const float su = sigmoid(o[0]), sr = sigmoid(o[1]);
    const float sp = fmaxf(o[0], 0.f) + log1pf(expf(-fabsf(o[0])));  // softplus(o0)
    const float er = sr - y[1], ep = o[2] - y[2];
    l += (double)(sp - y[0] * o[0]) + (double)wd * (double)er * (double)er + (double)wp * (double)ep * (double)ep;
    float* g = dO + (int64_t)i * kHeads;
    g[0] = (su - y[0]) * inv;
    g[1] = 2.f * wd * er * sr * (1.f - sr) * inv;
    g[2] = 2.f * wp * ep * inv;
  }
  __shared__ double s[kLossThreads];
  s[threadIdx.x] = l;
  __syncthreads();
  for (int w = kLossThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// loss_out = (sum of the block partials in order) / rows
__global__ void k_loss_final(const double* __restrict__ part, int nb, int rows, double* __restrict__ loss_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int q = 0; q < nb; q++) s += part[q];
  *loss_out = s / (double)rows;
}

// dH *= [H > 0] (H = relu(Z), kept in FP32)
__global__ void k_relu_back(int64_t total, const float* __restrict__ H, float* __restrict__ dH) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += step)
    if (!(H[e] > 0.f)) dH[e] = 0.f;
}

// part[y][j] = sum of dZ[i][j] over the rows of chunk y (blockIdx.y).  Block
// 32 x 8: the 8 threads of a column sum interleaved rows, then in order.
__global__ void __launch_bounds__(256) k_colsum_part(int rows, int N, const float* __restrict__ dZ,
                                                     float* __restrict__ part) {
  __shared__ float s[8][33];
  const int j = blockIdx.x * 32 + threadIdx.x;
  const int chunk = (rows + gridDim.y - 1) / gridDim.y;
  const int r0 = blockIdx.y * chunk, r1 = min(rows, r0 + chunk);
  float a = 0.f;
  if (j < N)
    for (int i = r0 + threadIdx.y; i < r1; i += 8) a += dZ[(int64_t)i * N + j];
  s[threadIdx.y][threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.y == 0 && j < N) {
    float t = 0.f;
    for (int q = 0; q < 8; q++) t += s[q][threadIdx.x];
    part[(int64_t)blockIdx.y * N + j] = t;
  }
}

// Adam on FP32 master values; the BF16 copy (if any) is refreshed
__global__ void k_adam(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16* __restrict__ wb) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += step) {
    const float ge = g[e];
    const float me = b1 * m[e] + (1.f - b1) * ge;
    const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
    m[e] = me;
    v[e] = ve;
    const float wn = w[e] - lr * (me / c1) / (sqrtf(ve / c2) + eps);
    w[e] = wn;
    if (wb) wb[e] = __float2bfloat16_rn(wn);
  }
}

__global__ void k_to_bf16(int64_t n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += step) b[e] = __float2bfloat16_rn(a[e]);
}

// flag = 1 if some a[e] lies outside [0, hi)
__global__ void k_idx_check(const int32_t* __restrict__ a, int64_t cnt, int64_t hi, int* flag) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += step)
    if (a[e] < 0 || a[e] >= hi) atomicOr(flag, 1);
}

__global__ void k_iota(int n, int32_t* __restrict__ idx) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) idx[i] = i;
}

int grid_e(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 148 * 8));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 2-D tensor map of a row-major BF16 matrix [rows x cols] (cols contiguous,
// a multiple of 8) read in boxes of 64 columns x box_rows rows with
// 128-byte swizzle; rows past the end read as zero.
int bf16_tmap(CUtensorMap* map, const __nv_bfloat16* base, int64_t rows, int cols, int box_rows) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f) {
      set_error("cuTensorMapEncodeTiled is not available");
      return SCUC_E_CUDA;
    }
    encode = reinterpret_cast<EncodeTiledFn>(f);
  }
  const cuuint64_t dim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kTcKc, (cuuint32_t)box_rows};
  const cuuint32_t estride[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dim, stride,
                            box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for a %lld x %d BF16 matrix", (int)r, (long long)rows, cols);
    return SCUC_E_CUDA;
  }
  return SCUC_OK;
}

}  // namespace

struct Mlp {
  int nl = 0;
  std::vector<int> dims;
  cudaStream_t s = nullptr;
  int device = 0;
  std::vector<float*> W, b, gW, gb, mW, vW, mb, vb;
  std::vector<__nv_bfloat16*> Wb;
  std::vector<__nv_bfloat16*> Wt;  // W_l^T (BF16, N x K) of the layers on tcgen05, else null
  int* tc_err = nullptr;           // bounded waits of k_gemm_tc that ran out
  int gemm_kind = 0;               // 0: tcgen05 for the eligible layers, 1: mma.sync for all
  float *mean = nullptr, *scale = nullptr;
  // activations for up to cap rows; activation gradients for up to tcap rows
  std::vector<float*> Z;
  std::vector<__nv_bfloat16*> Hb;
  std::vector<float*> dZ;
  float *Xs = nullptr, *Yb = nullptr, *dO = nullptr, *split = nullptr, *cpart = nullptr;
  double *part = nullptr, *loss_d = nullptr;
  int32_t* iota = nullptr;
  int* flag = nullptr;
  int cap = 0, tcap = 0, loss_cap = 0, iota_cap = 0;
  int64_t adam_t = 0;
  std::vector<void*> allocs;

  ~Mlp() {
    if (s) cudaStreamSynchronize(s);
    for (void* p : allocs) dev_free(p);
  }
  template <typename T>
  int alloc(T** p, size_t count) {
    void* q = nullptr;
    SCUC_TRY(dev_alloc_bytes(&q, std::max<size_t>(count, 1) * sizeof(T)));
    allocs.push_back(q);
    *p = static_cast<T*>(q);
    return SCUC_OK;
  }
  // release the buffers in `old` (after the stream has drained)
  int release(std::vector<void*> old) {
    SCUC_CUDA(cudaStreamSynchronize(s));
    for (void* p : old) {
      auto it = std::find(allocs.begin(), allocs.end(), p);
      if (it != allocs.end()) {
        allocs.erase(it);
        dev_free(p);
      }
    }
    return SCUC_OK;
  }
  int64_t nparams() const {
    int64_t c = 0;
    for (int l = 0; l < nl; l++) c += (int64_t)dims[l] * dims[l + 1] + dims[l + 1];
    return c;
  }
  int width_max() const { return *std::max_element(dims.begin(), dims.end()); }

  int ensure(int rows, bool train) {
    if (rows > cap) {
      std::vector<void*> old;
      for (void* p : Z) old.push_back(p);
      for (void* p : Hb) old.push_back(p);
      if (Xs) old.push_back(Xs);
      SCUC_TRY(release(old));
      Z.assign(nl, nullptr);
      Hb.assign(nl, nullptr);
      for (int l = 0; l < nl; l++) {
        SCUC_TRY(alloc(&Z[l], (size_t)rows * dims[l + 1]));
        SCUC_TRY(alloc(&Hb[l], (size_t)rows * dims[l + 1]));
      }
      SCUC_TRY(alloc(&Xs, (size_t)rows * dims[0]));
      cap = rows;
    }
    if (train && rows > tcap) {
      std::vector<void*> old;
      for (void* p : dZ) old.push_back(p);
      for (void* p : {(void*)Yb, (void*)dO, (void*)split, (void*)cpart})
        if (p) old.push_back(p);
      SCUC_TRY(release(old));
      dZ.assign(nl, nullptr);
      for (int l = 0; l < nl; l++) SCUC_TRY(alloc(&dZ[l], (size_t)rows * dims[l + 1]));
      SCUC_TRY(alloc(&Yb, (size_t)rows * kHeads));
      SCUC_TRY(alloc(&dO, (size_t)rows * kHeads));
      const int wm = width_max();
      SCUC_TRY(alloc(&split, (size_t)kSplitMax * wm * wm));
      SCUC_TRY(alloc(&cpart, (size_t)kColParts * wm));
      if (!part) SCUC_TRY(alloc(&part, kLossBlocks));
      tcap = rows;
    }
    return SCUC_OK;
  }
  int ensure_losses(int steps) {
    if (steps > loss_cap) {
      if (loss_d) SCUC_TRY(release({(void*)loss_d}));
      SCUC_TRY(alloc(&loss_d, (size_t)steps));
      loss_cap = steps;
    }
    return SCUC_OK;
  }
  int ensure_iota(int rows) {
    if (rows > iota_cap) {
      if (iota) SCUC_TRY(release({(void*)iota}));
      SCUC_TRY(alloc(&iota, (size_t)rows));
      k_iota<<<grid_e(rows), 256, 0, s>>>(rows, iota);
      SCUC_CUDA(cudaGetLastError());
      iota_cap = rows;
    }
    return SCUC_OK;
  }

  // layers whose forward product runs on tcgen05: BF16 input (not the
  // first layer), K a multiple of 64 up to 256, N a multiple of 16 up to 256
  bool tc_layer(int l) const {
    const int K = dims[l], N = dims[l + 1];
    return l > 0 && K % kTcKc == 0 && K <= kTcMaxK && N % 16 == 0 && N >= 16 && N <= kTcMaxN;
  }
  static uint32_t tmem_cols(int N) {
    uint32_t c = 32;
    while ((int)c < N) c <<= 1;
    return c;
  }
  int forward_tc(int l, int rows, bool keep_z) {
    const int K = dims[l], N = dims[l + 1];
    k_transpose_bf16<<<grid_e((int64_t)K * N), 256, 0, s>>>(K, N, Wb[l], Wt[l]);
    CUtensorMap th, tw;
    SCUC_TRY(bf16_tmap(&th, Hb[l - 1], rows, K, kTcM));
    SCUC_TRY(bf16_tmap(&tw, Wt[l], N, K, N));
    const int smem = 1024 + (K / kTcKc) * (kTcM * 128 + N * 128);
    SCUC_CUDA(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_gemm_tc<<<(rows + kTcM - 1) / kTcM, kTcThreads, smem, s>>>(th, tw, rows, N, K, tmem_cols(N), b[l],
                                                                  l < nl - 1 ? 1 : 0,
                                                                  keep_z || l == nl - 1 ? Z[l] : nullptr,
                                                                  l < nl - 1 ? Hb[l] : nullptr, tc_err);
    SCUC_CUDA(cudaGetLastError());
    return SCUC_OK;
  }
  // after the stream has drained: a bounded wait of k_gemm_tc that ran out
  int tc_check() {
    int e = 0;
    SCUC_CUDA(cudaMemcpyAsync(&e, tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCUC_CUDA(cudaStreamSynchronize(s));
    if (e) {
      SCUC_CUDA(cudaMemsetAsync(tc_err, 0, sizeof(int), s));
      set_error("tensor-core GEMM: a TMA or MMA completion wait ran out (flags %d)", e);
      return SCUC_E_DEVICE_TIMEOUT;
    }
    return SCUC_OK;
  }

  // Z_l for every layer from the standardized input Xs; keep_z = false
  // (prediction) keeps only the BF16 activations of the hidden layers that
  // run on tcgen05 (their FP32 Z is needed by the backward pass only)
  int forward(int rows, bool keep_z = true) {
    for (int l = 0; l < nl; l++) {
      const int K = dims[l], N = dims[l + 1];
      const dim3 g((N + kTN - 1) / kTN, (rows + kTM - 1) / kTM, 1);
      if (gemm_kind == 0 && tc_layer(l)) {
        SCUC_TRY(forward_tc(l, rows, keep_z));  // bias and activation in its epilogue
        continue;
      }
      if (l == 0)
        k_gemm<float, __nv_bfloat16><<<g, kGemmThreads, 0, s>>>(rows, N, K, K, Xs, K, 1, Wb[l], N, 1, Z[l], N, 0);
      else
        k_gemm<__nv_bfloat16, __nv_bfloat16>
            <<<g, kGemmThreads, 0, s>>>(rows, N, K, K, Hb[l - 1], K, 1, Wb[l], N, 1, Z[l], N, 0);
      k_bias_act<<<grid_e((int64_t)rows * N), 256, 0, s>>>(rows, N, Z[l], b[l], l < nl - 1,
                                                            l < nl - 1 ? Hb[l] : nullptr);
    }
    SCUC_CUDA(cudaGetLastError());
    return SCUC_OK;
  }

  // gW, gb of the batch-mean loss (targets in Yb); the batch loss to *loss_dev
  int backward(int rows, float wd, float wp, double* loss_dev) {
    const int nb = std::min(kLossBlocks, (rows + kLossThreads - 1) / kLossThreads);
    k_loss<<<nb, kLossThreads, 0, s>>>(rows, Z[nl - 1], Yb, wd, wp, dO, part);
    k_loss_final<<<1, 32, 0, s>>>(part, nb, rows, loss_dev);
    const float* dcur = dO;
    for (int l = nl - 1; l >= 0; l--) {
      const int K = dims[l], N = dims[l + 1];
      // gW_l = H_{l-1}^T dZ_l, the batch split into ns slices summed in order
      int ns = std::min(kSplitMax, std::max(1, rows / 256));
      const int kchunk = ((rows + ns - 1) / ns + kTK - 1) / kTK * kTK;
      ns = (rows + kchunk - 1) / kchunk;
      const dim3 gw((N + kTN - 1) / kTN, (K + kTM - 1) / kTM, ns);
      const int64_t slice = (int64_t)K * N;
      float* out = ns > 1 ? split : gW[l];
      if (l == 0)
        k_gemm<float, float><<<gw, kGemmThreads, 0, s>>>(K, N, rows, kchunk, Xs, 1, K, dcur, N, 1, out, N, slice);
      else
        k_gemm<__nv_bfloat16, float>
            <<<gw, kGemmThreads, 0, s>>>(K, N, rows, kchunk, Hb[l - 1], 1, K, dcur, N, 1, out, N, slice);
      if (ns > 1) k_sum_slices<<<grid_e(slice), 256, 0, s>>>(slice, ns, slice, split, gW[l]);
      // gb_l = column sums of dZ_l
      const dim3 gc((N + 31) / 32, kColParts);
      k_colsum_part<<<gc, dim3(32, 8), 0, s>>>(rows, N, dcur, cpart);
      k_sum_slices<<<grid_e(N), 256, 0, s>>>(N, kColParts, N, cpart, gb[l]);
      if (l > 0) {
        // dH_{l-1} = dZ_l W_l^T, then the ReLU mask of layer l-1
        const dim3 gh((K + kTN - 1) / kTN, (rows + kTM - 1) / kTM, 1);
        k_gemm<float, __nv_bfloat16>
            <<<gh, kGemmThreads, 0, s>>>(rows, K, N, N, dcur, N, 1, Wb[l], 1, N, dZ[l - 1], K, 0);
        k_relu_back<<<grid_e((int64_t)rows * K), 256, 0, s>>>((int64_t)rows * K, Z[l - 1], dZ[l - 1]);
        dcur = dZ[l - 1];
      }
    }
    SCUC_CUDA(cudaGetLastError());
    return SCUC_OK;
  }

  int adam(const scuc_ws_train_params& p) {
    adam_t++;
    const float c1 = 1.f - powf(p.beta1, (float)adam_t), c2 = 1.f - powf(p.beta2, (float)adam_t);
    for (int l = 0; l < nl; l++) {
      const int64_t nw = (int64_t)dims[l] * dims[l + 1];
      k_adam<<<grid_e(nw), 256, 0, s>>>(nw, W[l], gW[l], mW[l], vW[l], p.lr, p.beta1, p.beta2, p.eps, c1, c2, Wb[l]);
      k_adam<<<grid_e(dims[l + 1]), 256, 0, s>>>(dims[l + 1], b[l], gb[l], mb[l], vb[l], p.lr, p.beta1, p.beta2,
                                                 p.eps, c1, c2, nullptr);
    }
    SCUC_CUDA(cudaGetLastError());
    return SCUC_OK;
  }

  int standardize(int rows, const float* X, const int32_t* idx, const float* Y) {
    k_standardize<<<grid_e((int64_t)rows * dims[0]), 256, 0, s>>>(rows, dims[0], X, idx, mean, scale, Xs, Y,
                                                                  Y ? Yb : nullptr);
    SCUC_CUDA(cudaGetLastError());
    return SCUC_OK;
  }

  int clear_moments() {
    for (int l = 0; l < nl; l++) {
      const size_t nw = (size_t)dims[l] * dims[l + 1], nb = dims[l + 1];
      SCUC_CUDA(cudaMemsetAsync(mW[l], 0, nw * sizeof(float), s));
      SCUC_CUDA(cudaMemsetAsync(vW[l], 0, nw * sizeof(float), s));
      SCUC_CUDA(cudaMemsetAsync(mb[l], 0, nb * sizeof(float), s));
      SCUC_CUDA(cudaMemsetAsync(vb[l], 0, nb * sizeof(float), s));
    }
    adam_t = 0;
    return SCUC_OK;
  }
};

}  // namespace scuc

struct scuc_ws {
  scuc::Mlp m;
};

namespace {

// makes the handle's device current for the duration of a call
struct DeviceGuard {
  int prev = -1;
  int rc = SCUC_OK;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) {
      scuc::set_error("cudaSetDevice(%d) failed", dev);
      rc = SCUC_E_CUDA;
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int check_train_params(const scuc_ws_train_params* p) {
  if (!p || !(p->lr > 0.f) || !(p->beta1 >= 0.f && p->beta1 < 1.f) || !(p->beta2 >= 0.f && p->beta2 < 1.f) ||
      !(p->eps > 0.f) || !(p->w_dispatch >= 0.f) || !(p->w_price >= 0.f)) {
    scuc::set_error("invalid training parameters");
    return SCUC_E_INVALID;
  }
  return SCUC_OK;
}

}  // namespace

using scuc::Mlp;

extern "C" {

void scuc_ws_default_train_params(scuc_ws_train_params* p) {
  if (!p) return;
  p->lr = 1e-3f;
  p->beta1 = 0.9f;
  p->beta2 = 0.999f;
  p->eps = 1e-8f;
  p->w_dispatch = 1.f;
  p->w_price = 1.f;
}

int scuc_ws_create(scuc_ws** out, int32_t nlayers, const int32_t* dims, void* cuda_stream) {
  if (!out || !dims || nlayers < 1 || nlayers > 16) {
    scuc::set_error("scuc_ws_create: invalid arguments");
    return SCUC_E_INVALID;
  }
  *out = nullptr;
  for (int l = 0; l <= nlayers; l++)
    if (dims[l] < 1 || dims[l] > 4096) {
      scuc::set_error("scuc_ws_create: layer width %d out of range 1..4096", dims[l]);
      return SCUC_E_INVALID;
    }
  if (dims[nlayers] != scuc::kHeads) {
    scuc::set_error("scuc_ws_create: the last width must be %d", scuc::kHeads);
    return SCUC_E_INVALID;
  }
  scuc_ws* w = new scuc_ws();
  Mlp& M = w->m;
  M.nl = nlayers;
  M.dims.assign(dims, dims + nlayers + 1);
  M.s = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&M.device) != cudaSuccess) {
    delete w;
    scuc::set_error("scuc_ws_create: no CUDA device");
    return SCUC_E_CUDA;
  }
  int rc = SCUC_OK;
  M.W.assign(nlayers, nullptr); M.b.assign(nlayers, nullptr);
  M.gW.assign(nlayers, nullptr); M.gb.assign(nlayers, nullptr);
  M.mW.assign(nlayers, nullptr); M.vW.assign(nlayers, nullptr);
  M.mb.assign(nlayers, nullptr); M.vb.assign(nlayers, nullptr);
  M.Wb.assign(nlayers, nullptr);
  M.Wt.assign(nlayers, nullptr);
  rc = M.alloc(&M.tc_err, 1);
  if (rc == SCUC_OK && cudaMemsetAsync(M.tc_err, 0, sizeof(int), M.s) != cudaSuccess) {
    scuc::set_error("scuc_ws_create: cudaMemsetAsync failed");
    rc = SCUC_E_CUDA;
  }
  for (int l = 0; l < nlayers && rc == SCUC_OK; l++) {
    if (M.tc_layer(l) && (rc = M.alloc(&M.Wt[l], (size_t)dims[l] * dims[l + 1]))) break;
    const size_t nw = (size_t)dims[l] * dims[l + 1], nb = dims[l + 1];
    if ((rc = M.alloc(&M.W[l], nw)) || (rc = M.alloc(&M.b[l], nb)) || (rc = M.alloc(&M.gW[l], nw)) ||
        (rc = M.alloc(&M.gb[l], nb)) || (rc = M.alloc(&M.mW[l], nw)) || (rc = M.alloc(&M.vW[l], nw)) ||
        (rc = M.alloc(&M.mb[l], nb)) || (rc = M.alloc(&M.vb[l], nb)) || (rc = M.alloc(&M.Wb[l], nw)))
      break;
    if (cudaMemsetAsync(M.W[l], 0, nw * 4, M.s) != cudaSuccess || cudaMemsetAsync(M.b[l], 0, nb * 4, M.s) != cudaSuccess ||
        cudaMemsetAsync(M.Wb[l], 0, nw * 2, M.s) != cudaSuccess) {
      scuc::set_error("scuc_ws_create: cudaMemsetAsync failed");
      rc = SCUC_E_CUDA;
    }
  }
  if (rc == SCUC_OK) rc = M.alloc(&M.mean, dims[0]);
  if (rc == SCUC_OK) rc = M.alloc(&M.scale, dims[0]);
  if (rc == SCUC_OK) {
    std::vector<float> z(dims[0], 0.f), o(dims[0], 1.f);
    if (cudaMemcpyAsync(M.mean, z.data(), dims[0] * 4, cudaMemcpyHostToDevice, M.s) != cudaSuccess ||
        cudaMemcpyAsync(M.scale, o.data(), dims[0] * 4, cudaMemcpyHostToDevice, M.s) != cudaSuccess ||
        cudaStreamSynchronize(M.s) != cudaSuccess) {
      scuc::set_error("scuc_ws_create: copying the input standardisation failed");
      rc = SCUC_E_CUDA;
    }
  }
  if (rc == SCUC_OK) rc = M.clear_moments();
  if (rc == SCUC_OK && cudaStreamSynchronize(M.s) != cudaSuccess) {
    scuc::set_error("scuc_ws_create: stream synchronisation failed");
    rc = SCUC_E_CUDA;
  }
  if (rc != SCUC_OK) {
    delete w;
    return rc;
  }
  *out = w;
  return SCUC_OK;
}

int scuc_ws_num_params(const scuc_ws* w, int64_t* count) {
  if (!w || !count) {
    scuc::set_error("scuc_ws_num_params: null argument");
    return SCUC_E_INVALID;
  }
  *count = w->m.nparams();
  return SCUC_OK;
}

int scuc_ws_set_params(scuc_ws* w, const float* params) {
  if (!w || !params) {
    scuc::set_error("scuc_ws_set_params: null argument");
    return SCUC_E_INVALID;
  }
  Mlp& M = w->m;
  for (int64_t i = 0; i < M.nparams(); i++)
    if (!std::isfinite(params[i])) {
      scuc::set_error("scuc_ws_set_params: parameter %lld is not finite", (long long)i);
      return SCUC_E_INVALID;
    }
  DeviceGuard dg(M.device);
  SCUC_TRY(dg.rc);
  size_t off = 0;
  for (int l = 0; l < M.nl; l++) {
    const size_t nw = (size_t)M.dims[l] * M.dims[l + 1], nb = M.dims[l + 1];
    SCUC_CUDA(cudaMemcpyAsync(M.W[l], params + off, nw * 4, cudaMemcpyHostToDevice, M.s));
    off += nw;
    SCUC_CUDA(cudaMemcpyAsync(M.b[l], params + off, nb * 4, cudaMemcpyHostToDevice, M.s));
    off += nb;
    scuc::k_to_bf16<<<scuc::grid_e(nw), 256, 0, M.s>>>(nw, M.W[l], M.Wb[l]);
    SCUC_CUDA(cudaGetLastError());
  }
  SCUC_TRY(M.clear_moments());
  SCUC_CUDA(cudaStreamSynchronize(M.s));
  return SCUC_OK;
}

int scuc_ws_get_params(const scuc_ws* w, float* params) {
  if (!w || !params) {
    scuc::set_error("scuc_ws_get_params: null argument");
    return SCUC_E_INVALID;
  }
  const Mlp& M = w->m;
  DeviceGuard dg(M.device);
  SCUC_TRY(dg.rc);
  size_t off = 0;
  for (int l = 0; l < M.nl; l++) {
    const size_t nw = (size_t)M.dims[l] * M.dims[l + 1], nb = M.dims[l + 1];
    SCUC_CUDA(cudaMemcpyAsync(params + off, M.W[l], nw * 4, cudaMemcpyDeviceToHost, M.s));
    off += nw;
    SCUC_CUDA(cudaMemcpyAsync(params + off, M.b[l], nb * 4, cudaMemcpyDeviceToHost, M.s));
    off += nb;
  }
  SCUC_CUDA(cudaStreamSynchronize(M.s));
  return SCUC_OK;
}

int scuc_ws_set_input_norm(scuc_ws* w, const float* mean, const float* scale) {
  if (!w || !mean || !scale) {
    scuc::set_error("scuc_ws_set_input_norm: null argument");
    return SCUC_E_INVALID;
  }
  Mlp& M = w->m;
  for (int f = 0; f < M.dims[0]; f++)
    if (!std::isfinite(mean[f]) || !(scale[f] > 0.f) || !std::isfinite(scale[f])) {
      scuc::set_error("scuc_ws_set_input_norm: feature %d has mean %g, scale %g", f, mean[f], scale[f]);
      return SCUC_E_INVALID;
    }
  DeviceGuard dg(M.device);
  SCUC_TRY(dg.rc);
  SCUC_CUDA(cudaMemcpyAsync(M.mean, mean, M.dims[0] * 4, cudaMemcpyHostToDevice, M.s));
  SCUC_CUDA(cudaMemcpyAsync(M.scale, scale, M.dims[0] * 4, cudaMemcpyHostToDevice, M.s));
  SCUC_CUDA(cudaStreamSynchronize(M.s));
  return SCUC_OK;
}

int scuc_ws_predict(scuc_ws* w, const float* X_dev, int32_t rows, float* out_dev) {
  if (!w || rows < 0 || (rows > 0 && (!X_dev || !out_dev))) {
    scuc::set_error("scuc_ws_predict: invalid arguments");
    return SCUC_E_INVALID;
  }
  if (rows == 0) return SCUC_OK;
  Mlp& M = w->m;
  DeviceGuard dg(M.device);
  SCUC_TRY(dg.rc);
  SCUC_TRY(M.ensure(rows, false));
  SCUC_TRY(M.standardize(rows, X_dev, nullptr, nullptr));
  SCUC_TRY(M.forward(rows, false));
  scuc::k_heads<<<scuc::grid_e(rows), 256, 0, M.s>>>(rows, M.Z[M.nl - 1], out_dev);
  SCUC_CUDA(cudaGetLastError());
  SCUC_CUDA(cudaStreamSynchronize(M.s));
  return M.tc_check();
}

int scuc_ws_gradients(scuc_ws* w, const float* X_dev, const float* Y_dev, int32_t rows,
                      const scuc_ws_train_params* p, float* grads, double* loss) {
  if (!w || !X_dev || !Y_dev || rows <= 0) {
    scuc::set_error("scuc_ws_gradients: invalid arguments");
    return SCUC_E_INVALID;
  }
  SCUC_TRY(check_train_params(p));
  Mlp& M = w->m;
  DeviceGuard dg(M.device);
  SCUC_TRY(dg.rc);
  SCUC_TRY(M.ensure(rows, true));
  SCUC_TRY(M.ensure_losses(1));
  SCUC_TRY(M.ensure_iota(rows));
  SCUC_TRY(M.standardize(rows, X_dev, M.iota, Y_dev));
  SCUC_TRY(M.forward(rows));
  SCUC_TRY(M.backward(rows, p->w_dispatch, p->w_price, M.loss_d));
  if (loss) SCUC_CUDA(cudaMemcpyAsync(loss, M.loss_d, sizeof(double), cudaMemcpyDeviceToHost, M.s));
  if (grads) {
    size_t off = 0;
    for (int l = 0; l < M.nl; l++) {
      const size_t nw = (size_t)M.dims[l] * M.dims[l + 1], nb = M.dims[l + 1];
      SCUC_CUDA(cudaMemcpyAsync(grads + off, M.gW[l], nw * 4, cudaMemcpyDeviceToHost, M.s));
      off += nw;
      SCUC_CUDA(cudaMemcpyAsync(grads + off, M.gb[l], nb * 4, cudaMemcpyDeviceToHost, M.s));
      off += nb;
    }
  }
  SCUC_CUDA(cudaStreamSynchronize(M.s));
  return M.tc_check();
}

int scuc_ws_train(scuc_ws* w, const float* X_dev, const float* Y_dev, int64_t nsamples, const int32_t* idx_dev,
                  int32_t batch, int32_t steps, const scuc_ws_train_params* p, double* losses) {
  if (!w || !X_dev || !Y_dev || !idx_dev || nsamples <= 0 || batch <= 0 || steps < 0) {
    scuc::set_error("scuc_ws_train: invalid arguments");
    return SCUC_E_INVALID;
  }
  SCUC_TRY(check_train_params(p));
  if (steps == 0) return SCUC_OK;
  Mlp& M = w->m;
  DeviceGuard dg(M.device);
  SCUC_TRY(dg.rc);
  SCUC_TRY(M.ensure(batch, true));
  SCUC_TRY(M.ensure_losses(steps));
  // every sample index is checked before any kernel reads through it
  if (!M.flag) SCUC_TRY(M.alloc(&M.flag, 1));
  SCUC_CUDA(cudaMemsetAsync(M.flag, 0, sizeof(int), M.s));
  const int64_t nidx = (int64_t)batch * steps;
  scuc::k_idx_check<<<scuc::grid_e(nidx), 256, 0, M.s>>>(idx_dev, nidx, nsamples, M.flag);
  SCUC_CUDA(cudaGetLastError());
  int bad = 0;
  SCUC_CUDA(cudaMemcpyAsync(&bad, M.flag, sizeof(int), cudaMemcpyDeviceToHost, M.s));
  SCUC_CUDA(cudaStreamSynchronize(M.s));
  if (bad) {
    scuc::set_error("scuc_ws_train: a sample index is outside [0, %lld)", (long long)nsamples);
    return SCUC_E_INVALID;
  }
  for (int st = 0; st < steps; st++) {
    SCUC_TRY(M.standardize(batch, X_dev, idx_dev + (int64_t)st * batch, Y_dev));
    SCUC_TRY(M.forward(batch));
    SCUC_TRY(M.backward(batch, p->w_dispatch, p->w_price, M.loss_d + st));
    SCUC_TRY(M.adam(*p));
  }
  if (losses) SCUC_CUDA(cudaMemcpyAsync(losses, M.loss_d, steps * sizeof(double), cudaMemcpyDeviceToHost, M.s));
  SCUC_CUDA(cudaStreamSynchronize(M.s));
  return M.tc_check();
}

int scuc_ws_set_gemm(scuc_ws* w, int32_t kind) {
  if (!w || (kind != SCUC_WS_GEMM_TCGEN05 && kind != SCUC_WS_GEMM_MMA_SYNC)) {
    scuc::set_error("scuc_ws_set_gemm: invalid arguments");
    return SCUC_E_INVALID;
  }
  w->m.gemm_kind = kind;
  return SCUC_OK;
}

void scuc_ws_destroy(scuc_ws* w) {
  if (!w) return;
  DeviceGuard dg(w->m.device);
  cudaStreamSynchronize(w->m.s);
  delete w;
}

}  // extern "C"
