// Setup kernels: transpose, Pock-Chambolle scaling (Sec. 3.A), norms, power
// method for lambda_max(A A^T) (Sec. 3), iterate initialisation and output.
#pragma once
#include "lp_kernels.cuh"

namespace scuc {
namespace {  // internal linkage: each translation unit compiles its own copy


// ----------------------------- transpose ---------------------------------
__global__ void k_count_cols(const int* __restrict__ col, int64_t nnz, int* __restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
    atomicAdd(cnt + col[e], 1);
}

// one warp per row: entries of row i go to their column's next free slot
__global__ void k_scatter_t(const int* __restrict__ rp, const int* __restrict__ col, int m,
                            int* __restrict__ cursor, int* __restrict__ colt, int* __restrict__ permt) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = warp; i < m; i += nw)
    for (int e = rp[i] + lane; e < rp[i + 1]; e += 32) {
      const int pos = atomicAdd(cursor + col[e], 1);
      colt[pos] = i;
      permt[pos] = e;
    }
}

// sort the entries of short columns by row (thread per column, insertion)
__global__ void k_sort_small(const int* __restrict__ rpt, int n, int* __restrict__ colt,
                             int* __restrict__ permt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int a = rpt[j], b = rpt[j + 1];
  if (b - a > 32) return;
  for (int p = a + 1; p < b; p++) {
    const int kr = colt[p], kp = permt[p];
    int q = p - 1;
    while (q >= a && colt[q] > kr) {
      colt[q + 1] = colt[q];
      permt[q + 1] = permt[q];
      q--;
    }
    colt[q + 1] = kr;
    permt[q + 1] = kp;
  }
}

// sort the entries of one longer column (<= kSortCap) by row: bitonic in smem
constexpr int kSortCap = 8192;
__global__ void __launch_bounds__(1024) k_sort_block(const int* __restrict__ rpt, const int* __restrict__ cols,
                                                     int* __restrict__ colt, int* __restrict__ permt) {
  extern __shared__ unsigned long long keys[];
  const int j = cols[blockIdx.x];
  const int a = rpt[j], L = rpt[j + 1] - a;
  int P = 1;
  while (P < L) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x)
    keys[i] = i < L ? (((unsigned long long)(unsigned)colt[a + i]) << 32) | (unsigned)permt[a + i]
                    : ~0ull;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1)
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ jj;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const unsigned long long u = keys[i], v = keys[ixj];
          if ((u > v) == up) { keys[i] = v; keys[ixj] = u; }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    colt[a + i] = (int)(keys[i] >> 32);
    permt[a + i] = (int)(keys[i] & 0xffffffffu);
  }
}

__global__ void k_gather_t(const int* __restrict__ permt, int64_t nnz, const double* __restrict__ val,
                           double* __restrict__ valt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
    valt[e] = val[permt[e]];
}

// ------------------------- scan (exclusive) ------------------------------
constexpr int kScan = 1024;
__global__ void __launch_bounds__(kScan) k_scan_block(const int* __restrict__ in, int n, int* __restrict__ out,
                                                      int* __restrict__ bsum) {
  __shared__ int ws[kScan / 32];
  const int i = blockIdx.x * kScan + threadIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int v = i < n ? in[i] : 0;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    ws[lane] = s;
  }
  __syncthreads();
  const int incl = x + (w > 0 ? ws[w - 1] : 0);
  if (i < n) out[i] = incl - v;
  if (threadIdx.x == kScan - 1) bsum[blockIdx.x] = incl;
}

__global__ void k_scan_add(int* __restrict__ out, int n, const int* __restrict__ boff) {
  const int i = blockIdx.x * kScan + threadIdx.x;
  if (i < n) out[i] += boff[blockIdx.x];
}

// out[n] = the total
__global__ void k_scan_total(const int* __restrict__ in, int n, int* __restrict__ out) {
  if (threadIdx.x == 0) out[n] = n > 0 ? in[n - 1] + out[n - 1] : 0;
}

// --------------------------- scaling -------------------------------------
__global__ void k_fill(double* __restrict__ a, int na, double* __restrict__ b, int nb, double v) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na; i += stride) a[i] = v;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += stride) b[i] = v;
}

// Factor of one scaling pass for each row of a CSR (thread per row,
// sequential in entry order): 1/sqrt(max) (Ruiz) or 1/sqrt(sum) (Pock-
// Chambolle) of |(Dr[row] * a) * Dc[col]| over the row, 1 for empty rows.
// transposed = 1: the CSR is A^T (rows are columns of A).  The solver runs
// it for the Ruiz passes; its sum passes run as products (k_abs2 +
// k_factor_from_sums), which balance the long rows.
__global__ void k_scale_factor(const int* __restrict__ rp, const int* __restrict__ col,
                               const double* __restrict__ val, int m, const double* __restrict__ Dr,
                               const double* __restrict__ Dc, int transposed, int use_max,
                               double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = 0.0;
  for (int e = rp[i]; e < rp[i + 1]; e++) {
    const double a = transposed ? fabs((Dr[col[e]] * val[e]) * Dc[i]) : fabs((Dr[i] * val[e]) * Dc[col[e]]);
    if (use_max) s = a > s ? a : s;
    else s += a;
  }
  out[i] = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
}

// |a| and |b| elementwise (the absolute matrix values of a sum pass)
__global__ void k_abs2(const double* __restrict__ a, double* __restrict__ oa, int64_t na,
                       const double* __restrict__ b, double* __restrict__ ob, int64_t nb) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na; i += stride) oa[i] = fabs(a[i]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += stride) ob[i] = fabs(b[i]);
}

// Factor of a sum pass from the row sums of |A| weighted by the other side's
// D: sum_j |D_i a_ij D'_j| = D_i sum_j |a_ij| D'_j (D > 0), so the factor is
// 1/sqrt(D_i * s_i), 1 for empty rows.  In place (out may be s).
__global__ void k_factor_from_sums(int m, const double* __restrict__ D, const double* s, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double v = D[i] * s[i];
  out[i] = v > 0.0 ? 1.0 / sqrt(v) : 1.0;
}

__global__ void k_mul2(double* __restrict__ a, const double* __restrict__ fa, int na, double* __restrict__ b,
                       const double* __restrict__ fb, int nb) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na; i += stride) a[i] *= fa[i];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += stride) b[i] *= fb[i];
}

// row sums in entry order, column sums in row order (sequential, one thread
// per row/column), then D = 1/sqrt(sum) (1 for empty rows/columns)
__global__ void k_abs_sum_inv_sqrt(const int* __restrict__ rp, const double* __restrict__ val, int m,
                                   int use_scaling, double* __restrict__ D) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  if (!use_scaling) { D[i] = 1.0; return; }
  double s = 0.0;
  for (int e = rp[i]; e < rp[i + 1]; e++) s += fabs(val[e]);
  D[i] = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
}

// vs[e] = (Dr[i] * val[e]) * Dc[col[e]]   (warp per row)
__global__ void k_scale_vals(const int* __restrict__ rp, const int* __restrict__ col,
                             const double* __restrict__ val, int m, const double* __restrict__ Dr,
                             const double* __restrict__ Dc, double* __restrict__ vs) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = warp; i < m; i += nw) {
    const double d = Dr[i];
    for (int e = rp[i] + lane; e < rp[i + 1]; e += 32) vs[e] = (d * val[e]) * Dc[col[e]];
  }
}

__global__ void k_scale_vecs(int m, int n, const double* __restrict__ Dr, const double* __restrict__ Dc,
                             const double* __restrict__ c, const double* __restrict__ xl,
                             const double* __restrict__ xu, const double* __restrict__ lo,
                             const double* __restrict__ hi, double* __restrict__ cs,
                             double* __restrict__ xls, double* __restrict__ xus,
                             double* __restrict__ los, double* __restrict__ his) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    cs[j] = Dc[j] * c[j];
    xls[j] = xl[j] / Dc[j];
    xus[j] = xu[j] / Dc[j];
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    los[i] = Dr[i] * lo[i];
    his[i] = Dr[i] * hi[i];
  }
}

__device__ __forceinline__ double bound_mag(double lo, double hi) {
  double b = 0.0;
  if (isfinite(lo) && fabs(lo) > b) b = fabs(lo);
  if (isfinite(hi) && fabs(hi) > b) b = fabs(hi);
  return b;
}

// stage 1 of the four norms: {sum bmag(los,his)^2, sum cs^2, sum bmag(lo,hi)^2, sum c^2}
constexpr int kNormBlocks = 592;  // 4 x 148 SMs
__global__ void __launch_bounds__(kBlock) k_norms_partial(int m, int n, const double* __restrict__ los,
                                                          const double* __restrict__ his,
                                                          const double* __restrict__ cs,
                                                          const double* __restrict__ lo,
                                                          const double* __restrict__ hi,
                                                          const double* __restrict__ c,
                                                          double* __restrict__ part) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const double a = bound_mag(los[i], his[i]);
    const double b = bound_mag(lo[i], hi[i]);
    v[0] += a * a;
    v[2] += b * b;
  }
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    v[1] += cs[j] * cs[j];
    v[3] += c[j] * c[j];
  }
  block_store<4>(v, part, gridDim.x);
}

// stage 2: beta = 1 + ||b_hat||, gamma = 1 + ||c_hat|| (1 when unscaled),
// bnorm = ||b||, cnorm = ||c|| of the unscaled LP
__global__ void __launch_bounds__(kDecideThreads) k_norms_final(const double* __restrict__ part, int nb,
                                                                int use_scaling, Ctrl* C) {
  const double b2 = decide_sum(part + 0 * nb, nb);
  const double c2 = decide_sum(part + 1 * nb, nb);
  const double ub2 = decide_sum(part + 2 * nb, nb);
  const double uc2 = decide_sum(part + 3 * nb, nb);
  if (threadIdx.x == 0) {
    C->beta = use_scaling ? 1.0 + sqrt(b2) : 1.0;
    C->gamma = use_scaling ? 1.0 + sqrt(c2) : 1.0;
    C->bnorm = sqrt(ub2);
    C->cnorm = sqrt(uc2);
  }
}

__global__ void k_normalize(int m, int n, const Ctrl* __restrict__ C, double* __restrict__ cs,
                            double* __restrict__ xls, double* __restrict__ xus,
                            double* __restrict__ los, double* __restrict__ his) {
  const double beta = C->beta, gamma = C->gamma;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    xls[j] /= beta;
    xus[j] /= beta;
    cs[j] /= gamma;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    los[i] /= beta;
    his[i] /= beta;
  }
}

__global__ void k_to_f32(const double* __restrict__ a, int64_t k, float* __restrict__ b) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < k; e += stride) b[e] = (float)a[e];
}

// Values of the sliced ELL copy (Sell) from the CSR arrays of the same
// matrix: one warp per slice, lane r copies its row's entries in order and
// pads the slice with its last column and zero.  FP32 values (v32 != null)
// go to cv32 with their columns, or, in the compressed form, to v2 with the
// 16-bit offsets from the entry's cluster base in o2 (S.lrec filled by
// k_sell_lrec); FP64 values (v64 != null) to col / v64.
__global__ void __launch_bounds__(kBlock) k_sell_fill(Sell S, const int* __restrict__ rp,
                                                      const int* __restrict__ col, const double* __restrict__ v64,
                                                      const float* __restrict__ v32) {
  const int sl = (int)blockIdx.x * (kBlock / 32) + (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (sl >= S.nslice) return;
  const int r = S.rows[(size_t)sl * 32 + lane];
  const int a = r >= 0 ? rp[r] : 0, len = r >= 0 ? rp[r + 1] - a : 0;
  const int last = len > 0 ? col[a + len - 1] : 0;
  const int steps = S.sptr[sl + 1] - S.sptr[sl];
  const int64_t base = (int64_t)S.sptr[sl] * 32 + lane;
  for (int k = 0; k < steps; k++) {
    const int64_t e = base + (int64_t)k * 32;
    const bool in = k < len;
    const int c = in ? col[a + k] : last;
    if (v32 && !S.compressed) S.cv32[e] = make_int2(c, __float_as_int(in ? v32[a + k] : 0.0f));
    if (v64) {
      S.col[e] = c;
      S.v64[e] = in ? v64[a + k] : 0.0;
    }
  }
  if (v32 && S.compressed) {
    const int4 rec = S.lrec[(size_t)sl * 32 + lane];
    const int np = S.pptr[sl + 1] - S.pptr[sl];
    const int64_t pb = (int64_t)S.pptr[sl] * 32 + lane;
    for (int p = 0; p < np; p++) {
      float v[2];
      unsigned o[2];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int k = 2 * p + h;
        const bool in = k < len;
        const int c = in ? col[a + k] : last;
        v[h] = in ? v32[a + k] : 0.0f;
        o[h] = (unsigned)(c - (k < rec.w ? rec.y : rec.z));
      }
      S.v2[pb + (int64_t)p * 32] = make_float2(v[0], v[1]);
      S.o2[pb + (int64_t)p * 32] = (o[0] & 0xffffu) | (o[1] << 16);
    }
  }
}

// Cluster bases of the compressed FP32 form (Sell::lrec): lane r of a slice
// splits its row's columns (sorted) at the first one more than kSpan16 past
// the row's first column; *bad is set if the second part spans more than
// kSpan16 as well (the copy then keeps the 32-bit form).  Lanes without a
// row, and empty rows, get base 0.
__global__ void __launch_bounds__(kBlock) k_sell_lrec(Sell S, const int* __restrict__ rp,
                                                      const int* __restrict__ col, int* __restrict__ bad) {
  const int sl = (int)blockIdx.x * (kBlock / 32) + (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (sl >= S.nslice) return;
  const int r = S.rows[(size_t)sl * 32 + lane];
  const int a = r >= 0 ? rp[r] : 0, len = r >= 0 ? rp[r + 1] - a : 0;
  int b0 = len > 0 ? col[a] : 0, b1 = b0, kj = len;
  for (int k = 1; k < len; k++) {
    const int c = col[a + k];
    if (kj == len) {
      if ((int64_t)c - b0 > kSpan16) {
        kj = k;
        b1 = c;
      }
    } else if ((int64_t)c - b1 > kSpan16) {
      *bad = 1;
      break;
    }
  }
  S.lrec[(size_t)sl * 32 + lane] = make_int4(r, b0, b1, kj);
}

// Column part of the FP32 chunk stream (Partition::cst / crec), once per
// handle: one warp per chunk; the chunk's columns (sorted) split at the
// first one more than kSpan16 past the first column; a chunk whose second
// part spans more than kSpan16 as well gets base0 = -1 (32-bit columns).
// Padding entries repeat the last entry's offset.  *n16 counts the entries
// of the chunks that use offsets.
__global__ void __launch_bounds__(kBlock) k_chunk_rec(const int* __restrict__ col, Partition P,
                                                      unsigned long long* __restrict__ n16) {
  const int w = (int)blockIdx.x * (kBlock / 32) + (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= P.nchunk) return;
  const int2 c = P.chunks[w];
  const int len = c.y - c.x;
  const int b0 = col[c.x];
  int split = len;
  for (int i = lane; i < len; i += 32)
    if ((int64_t)col[c.x + i] - b0 > kSpan16) {
      split = i;
      break;
    }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) split = min(split, __shfl_xor_sync(0xffffffffu, split, off));
  const int b1 = split < len ? col[c.x + split] : b0;
  const bool narrow = (int64_t)col[c.y - 1] - b1 <= kSpan16;
  unsigned short* offs = reinterpret_cast<unsigned short*>(P.cst + (size_t)w * kChunkRec16) + 2 * kChunk;
  for (int i = lane; narrow && i < kChunk; i += 32) {
    const int e = c.x + min(i, len - 1);
    offs[i] = (unsigned short)(col[e] - (min(i, len - 1) < split ? b0 : b1));
  }
  if (lane == 0) {
    P.crec[w] = make_int4(narrow ? b0 : -1, b1, (len << 16) | split, 0);
    if (narrow) atomicAdd(n16, (unsigned long long)len);
  }
}

// Value part of the FP32 chunk stream, after every FP32 scaling: one warp
// per chunk copies its FP32 values, zero padded to kChunk.
__global__ void __launch_bounds__(kBlock) k_chunk_vals(const float* __restrict__ v32, Partition P) {
  const int w = (int)blockIdx.x * (kBlock / 32) + (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= P.nchunk) return;
  const int2 c = P.chunks[w];
  const int len = c.y - c.x;
  float* vals = reinterpret_cast<float*>(P.cst + (size_t)w * kChunkRec16);
  for (int i = lane; i < kChunk; i += 32) vals[i] = i < len ? v32[c.x + i] : 0.0f;
}

// --------------------------- power method ---------------------------------
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t j) {
  uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void __launch_bounds__(kBlock) k_power_seed(int n, uint64_t seed, double* __restrict__ q,
                                                       double* __restrict__ part) {
  double v[1] = {0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const double a = 0.5 + (double)(splitmix64_at(seed, (uint64_t)j) >> 11) * 0x1.0p-53;
    q[j] = a;
    v[0] += a * a;
  }
  block_store<1>(v, part, gridDim.x);
}

__global__ void __launch_bounds__(kDecideThreads) k_power_seed_norm(const double* part, int nb, PowerCtrl* P) {
  const double s = decide_sum(part, nb);
  if (threadIdx.x == 0) P->nw = sqrt(s);
}

struct StoreEpi {  // out[r] = acc, and sum of squares
  double* out;
  double acc[1];
  __device__ void load(int) {}
  __device__ void row(int r, double a) {
    out[r] = a;
    acc[0] += a * a;
  }
};

__global__ void __launch_bounds__(kBlock) k_power_spmv(const int* __restrict__ rp, const int* __restrict__ col,
                                                       const double* __restrict__ val,
                                                       const double* __restrict__ in, Partition part,
                                                       double* __restrict__ out, double* __restrict__ psum,
                                                       const PowerCtrl* __restrict__ P) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (P->done) return;
  StoreEpi epi{out, {0.0}};
  spmv_block<double>(rp, col, val, in, part, smem, epi);
  block_store<1>(epi.acc, psum, part);
}

// FP32 products for MIXED solves (FP32 values and vectors, FP32 sums; the
// squares and norms in FP64): out32 = the product, out (may be null) its
// FP64 copy
struct StoreEpi32 {
  double* out;
  float* out32;
  double acc[1];
  __device__ void load(int) {}
  __device__ void row(int r, float a) {
    const double d = (double)a;
    if (out) out[r] = d;
    out32[r] = a;
    acc[0] += d * d;
  }
};

__global__ void __launch_bounds__(kBlock) k_power_spmv32(const int* __restrict__ rp, const int* __restrict__ col,
                                                         const float* __restrict__ val,
                                                         const float* __restrict__ in, Partition part,
                                                         double* __restrict__ out, float* __restrict__ out32,
                                                         double* __restrict__ psum, const PowerCtrl* __restrict__ P) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (P->done) return;
  StoreEpi32 epi{out, out32, {0.0}};
  spmv_block<float>(rp, col, val, in, part, smem, epi);
  block_store<1>(epi.acc, psum, part);
}

// Chunk launch of a power iteration: returns at once when the estimate has
// converged (a round queues 16 iterations; those after the last do nothing).
template <typename VT>
__global__ void __launch_bounds__(kBlock) k_power_chunks(const int* __restrict__ col, const VT* __restrict__ val,
                                                         const VT* __restrict__ x, Partition part,
                                                         const PowerCtrl* __restrict__ P) {
  if (P->done) return;
  chunk_warp<VT>(col, val, x, part);
}

// The A^T product of an FP32 power iteration on the sliced copy of A^T
// (one LP; its partial sums in A^T's CSR partition slots, as
// k_power_spmv32 stores them).
__global__ void __launch_bounds__(kBlock) k_power_sell32(Sell S, Partition pT, const float* __restrict__ in,
                                                         double* __restrict__ out, float* __restrict__ out32,
                                                         double* __restrict__ psum, const PowerCtrl* __restrict__ P) {
  if (P->done) return;
  StoreEpi32 epi{out, out32, {0.0}};
  sell_gridstride<float>(S, pT, in, epi);
  sell_store<1>(epi.acc, psum, pT.nblk);
}

__global__ void __launch_bounds__(kDecideThreads) k_power_decide(const double* pu, int nA, const double* pw,
                                                                 int nT, PowerCtrl* P) {
  if (P->done) return;
  const double lam = decide_sum(pu, nA);
  const double w2 = decide_sum(pw, nT);
  if (threadIdx.x != 0) return;
  P->it++;
  P->lam = lam;
  P->nw = sqrt(w2);
  // stop on a zero product, on a relative change <= tol, or at the limit
  if (P->nw == 0.0) P->done = 1;
  else if (P->it > 1 && fabs(lam - P->lam_prev) <= P->tol * lam) P->done = 1;
  else if (P->it >= P->max_iter) P->done = 1;
  P->lam_prev = lam;
}

// q = w / ||w||  (not needed once the estimate is final); q32 (may be null)
// its FP32 copy for FP32 products
__global__ void k_power_norm(int n, const double* __restrict__ w, double* __restrict__ q, float* __restrict__ q32,
                             const PowerCtrl* P) {
  if (P->done) return;
  const double nw = P->nw;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const double v = w[j] / nw;
    q[j] = v;
    if (q32) q32[j] = (float)v;
  }
}

__global__ void k_power_norm_seed(int n, double* __restrict__ q, float* __restrict__ q32, const PowerCtrl* P) {
  const double nq = P->nw;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const double v = q[j] / nq;
    q[j] = v;
    if (q32) q32[j] = (float)v;
  }
}

// ------------------------ iterate init / output ---------------------------
// blockIdx.y = LP of the batch
__global__ void k_init_iterates(DevLP L, const double* __restrict__ xin, const double* __restrict__ yin) {
  const int lp = blockIdx.y;
  if (blockIdx.x == 0 && threadIdx.x == 0) L.ctrl[lp].t_start_ns = globaltimer_ns();
  const double beta = L.ctrl[lp].beta, gamma = L.ctrl[lp].gamma;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int c0, c1, r0, r1;
  lp_range(L.col0, lp, L.n, c0, c1);
  lp_range(L.row0, lp, L.m, r0, r1);
  for (int64_t j = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < c1; j += stride) {
    const double v = xin ? xin[j] / (beta * L.Dc[j]) : 0.0;
    const double x = clampd(v, L.xl[j], L.xu[j]);
    L.x[j] = x;
    L.x0[j] = x;
  }
  for (int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r1; i += stride) {
    double v = yin ? yin[i] / (gamma * L.Dr[i]) : 0.0;
    if (!isfinite(L.lo[i]) && v > 0.0) v = 0.0;
    if (!isfinite(L.hi[i]) && v < 0.0) v = 0.0;
    L.y[i] = v;
    L.y0[i] = v;
    L.y32[i] = (float)v;
  }
}

// blockIdx.y = LP of the batch
// Outputs of the last check, unscaled; an infeasibility verdict returns its
// certificate instead (the ray y_bar - y in yo, or the direction x_bar - x
// in xo).
__global__ void k_finalize(DevLP L, double* __restrict__ xo, double* __restrict__ yo, double* __restrict__ zo) {
  const int lp = blockIdx.y;
  const double beta = L.ctrl[lp].beta, gamma = L.ctrl[lp].gamma;
  const int status = L.ctrl[lp].status;
  const double* xs = status == SCUC_ST_DUAL_INFEASIBLE ? L.dxchk : L.xbar;
  const double* ys = status == SCUC_ST_PRIMAL_INFEASIBLE ? L.dychk : L.ybar;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int c0, c1, r0, r1;
  lp_range(L.col0, lp, L.n, c0, c1);
  lp_range(L.row0, lp, L.m, r0, r1);
  for (int64_t j = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < c1; j += stride) {
    if (xo) xo[j] = beta * L.Dc[j] * xs[j];
    if (zo) zo[j] = gamma * L.zbar[j] / L.Dc[j];
  }
  if (yo)
    for (int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r1; i += stride)
      yo[i] = gamma * L.Dr[i] * ys[i];
}

// unscaled product (matvec entry point)
struct PlainEpi {
  double* out;
  __device__ void load(int) {}
  __device__ void row(int r, double a) { out[r] = a; }
};

__global__ void __launch_bounds__(kBlock) k_spmv_plain(const int* __restrict__ rp, const int* __restrict__ col,
                                                       const double* __restrict__ val,
                                                       const double* __restrict__ in, Partition part,
                                                       double* __restrict__ out) {
  extern __shared__ __align__(128) unsigned char smem[];
  PlainEpi epi{out};
  spmv_block<double>(rp, col, val, in, part, smem, epi);
}

}  // namespace

}  // namespace scuc
