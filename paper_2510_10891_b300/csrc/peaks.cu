// FMA throughput of the current GPU (scuc_probe_fma_peak in
// include/scuc_lp.h): the denominator of the rooflines of kernels bound by
// the FP64 pipe rather than by HBM.  Every thread runs eight independent
// register-resident FMA chains; the clocks are left as they are.
#include <cstdio>

#include "lp.h"

namespace scuc {
namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_loop(T* __restrict__ out, int iters, T a, T b) {
  T v[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) v[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < kChains; k++) v[k] = fma(v[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += v[k];
  if (s == (T)-12345.0) out[blockIdx.x] = s;  // never true: keeps the loop
}

template <typename T>
int measure(double* tflops, double* ms_out) {
  int dev = 0, sms = 0;
  SCUC_CUDA(cudaGetDevice(&dev));
  SCUC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = 1 << 14;
  T* out = nullptr;
  SCUC_CUDA(cudaMalloc(&out, blocks * sizeof(T)));
  cudaEvent_t e0, e1;
  SCUC_CUDA(cudaEventCreate(&e0));
  SCUC_CUDA(cudaEventCreate(&e1));
  // a = 1 - 2^-20, b = 2^-10: the chains converge to b / (1 - a) and stay finite
  const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1024.0);
  float best = 1e30f;
  int rc = SCUC_OK;
  for (int rep = 0; rep < 4 && rc == SCUC_OK; rep++) {  // first launch is warm-up
    cudaEventRecord(e0);
    k_fma_loop<T><<<blocks, threads>>>(out, iters, a, b);
    cudaEventRecord(e1);
    const cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      set_error("FMA probe: %s", cudaGetErrorString(e));
      rc = SCUC_E_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != SCUC_OK) return rc;
  const double flops = 2.0 * kChains * (double)iters * blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return SCUC_OK;
}

}  // namespace
}  // namespace scuc

extern "C" int scuc_probe_fma_peak(int32_t fp64, double* tflops, double* ms) {
  if (!tflops) {
    scuc::set_error("scuc_probe_fma_peak: null argument");
    return SCUC_E_INVALID;
  }
  return fp64 ? scuc::measure<double>(tflops, ms) : scuc::measure<float>(tflops, ms);
}
