// Warm-start network (scuc_ws_* in include/scuc_ws.h): a multilayer
// perceptron with hand-written forward, backward and Adam kernels.
//
// GEMMs run on the tensor cores (mma m16n8k16, BF16 operands, FP32
// accumulation); operands are converted to BF16 while they are staged in
// shared memory, so one kernel serves the forward product (X W), the weight
// gradient (H^T dZ, split over the batch) and the input gradient (dZ W^T).
// Master weights, biases and Adam moments are FP32.  Every reduction (batch
// loss, bias gradient, split-K partial products) has a fixed order, so
// training is deterministic.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/scuc_ws.h"
#include "common.cuh"

namespace scuc {
int dev_alloc_bytes(void** p, size_t bytes);

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

}  // namespace

struct Mlp {
  int nl = 0;
  std::vector<int> dims;
  cudaStream_t s = nullptr;
  int device = 0;
  std::vector<float*> W, b, gW, gb, mW, vW, mb, vb;
  std::vector<__nv_bfloat16*> Wb;
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
    for (void* p : allocs) cudaFree(p);
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
        cudaFree(p);
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

  // Z_l for every layer from the standardized input Xs
  int forward(int rows) {
    for (int l = 0; l < nl; l++) {
      const int K = dims[l], N = dims[l + 1];
      const dim3 g((N + kTN - 1) / kTN, (rows + kTM - 1) / kTM, 1);
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
  for (int l = 0; l < nlayers && rc == SCUC_OK; l++) {
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
  SCUC_TRY(M.forward(rows));
  scuc::k_heads<<<scuc::grid_e(rows), 256, 0, M.s>>>(rows, M.Z[M.nl - 1], out_dev);
  SCUC_CUDA(cudaGetLastError());
  SCUC_CUDA(cudaStreamSynchronize(M.s));
  return SCUC_OK;
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
  return SCUC_OK;
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
  return SCUC_OK;
}

void scuc_ws_destroy(scuc_ws* w) {
  if (!w) return;
  DeviceGuard dg(w->m.device);
  cudaStreamSynchronize(w->m.s);
  delete w;
}

}  // extern "C"
