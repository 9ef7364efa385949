// Elementwise kernels of the AB and Naive variants (Section 4.1):
//   block_sum - an explicit operand-sum temporary  X^ = sum_s delta_s X_s  (Naive),
//   combine   - the separate C updates  C_q += gamma_q M  after a product (AB, Naive).
// Both are grid-stride loops over rows with coalesced column access; each element of
// the destination is produced by exactly one thread, so the order of the additions
// is fixed (left to right over the terms).
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace sgb {
namespace {

struct SumParams {
  double* dst;
  int64_t rows, cols;
  const double* src;
  int64_t ld, src_rows, src_cols, h_r, h_c;
  int nterms;
  int trans;  // the source is stored transposed: element (r, c) at src[c * ld + r]
  uint8_t terms[kMaxTerms];
};

__global__ void block_sum_kernel(const __grid_constant__ SumParams p) {
  const int64_t total = p.rows * p.cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / p.cols, j = e - (e / p.cols) * p.cols;
    double v = 0.0;
    for (int t = 0; t < p.nterms; ++t) {
      const uint8_t c = p.terms[t];
      const int64_t gr = (int64_t)term_bi(c) * p.h_r + i, gc = (int64_t)term_bj(c) * p.h_c + j;
      double x = 0.0;
      if (i < p.h_r && j < p.h_c && gr < p.src_rows && gc < p.src_cols)
        x = p.trans ? p.src[gc * p.ld + gr] : p.src[gr * p.ld + gc];
      if (t == 0) v = term_neg(c) ? -x : x;
      else v = term_neg(c) ? v - x : v + x;
    }
    p.dst[e] = v;
  }
}

struct CombineParams {
  double* C;
  int64_t ldc, c_rows, c_cols;
  const double* M;
  int64_t hm, hn;
  double alpha;
  int ntargets;
  uint8_t targets[kMaxTerms];
};

__global__ void combine_kernel(const __grid_constant__ CombineParams p) {
  const int64_t total = p.hm * p.hn;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / p.hn, j = e - (e / p.hn) * p.hn;
    const double m = p.alpha == 1.0 ? p.M[e] : p.alpha * p.M[e];  // no FP64 multiply for alpha = 1
    for (int t = 0; t < p.ntargets; ++t) {
      const uint8_t c = p.targets[t];
      const int64_t gr = (int64_t)term_bi(c) * p.hm + i, gc = (int64_t)term_bj(c) * p.hn + j;
      if (gr < p.c_rows && gc < p.c_cols) {
        double* d = p.C + gr * p.ldc + gc;
        *d = term_neg(c) ? *d - m : *d + m;
      }
    }
  }
}

// C = beta C over the m x n operand (BLAS semantics: beta = 0 writes zeros without
// reading C).
__global__ void scale_kernel(double* C, int64_t ldc, int64_t rows, int64_t cols, double beta, int tri) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e - (e / cols) * cols;
    if ((tri == 1 && j > i) || (tri == 2 && j < i)) continue;
    double* d = C + i * ldc + j;
    *d = beta == 0.0 ? 0.0 : beta * *d;
  }
}

int grid_for(int64_t total, int threads) {
  const int64_t want = (total + threads - 1) / threads;
  const int64_t cap = (int64_t)std::max(device_sm_count(), 1) * 16;
  return (int)std::max<int64_t>(1, std::min(want, cap));
}

}  // namespace

cudaError_t launch_block_sum(double* dst, int64_t rows, int64_t cols, const double* src, int64_t ld,
                             int64_t src_rows, int64_t src_cols, int64_t h_r, int64_t h_c,
                             const uint8_t* terms, int nterms, cudaStream_t stream, int trans) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  if (nterms < 1 || nterms > kMaxTerms) return cudaErrorInvalidValue;
  SumParams p;
  p.dst = dst; p.rows = rows; p.cols = cols; p.src = src; p.ld = ld;
  p.src_rows = src_rows; p.src_cols = src_cols; p.h_r = h_r; p.h_c = h_c; p.nterms = nterms;
  p.trans = trans;
  for (int t = 0; t < kMaxTerms; ++t) p.terms[t] = t < nterms ? terms[t] : 0;
  const int threads = 256;
  block_sum_kernel<<<grid_for(rows * cols, threads), threads, 0, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_combine(double* C, int64_t ldc, int64_t c_rows, int64_t c_cols, const double* M,
                           int64_t hm, int64_t hn, const uint8_t* targets, int ntargets,
                           cudaStream_t stream, double alpha) {
  if (hm <= 0 || hn <= 0) return cudaSuccess;
  if (ntargets < 1 || ntargets > kMaxTerms) return cudaErrorInvalidValue;
  CombineParams p;
  p.C = C; p.ldc = ldc; p.c_rows = c_rows; p.c_cols = c_cols; p.M = M; p.hm = hm; p.hn = hn;
  p.alpha = alpha;
  p.ntargets = ntargets;
  for (int t = 0; t < kMaxTerms; ++t) p.targets[t] = t < ntargets ? targets[t] : 0;
  const int threads = 256;
  combine_kernel<<<grid_for(hm * hn, threads), threads, 0, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_scale(double* C, int64_t ldc, int64_t rows, int64_t cols, double beta, cudaStream_t stream,
                         int tri) {
  if (rows <= 0 || cols <= 0 || beta == 1.0) return cudaSuccess;
  const int threads = 256;
  scale_kernel<<<grid_for(rows * cols, threads), threads, 0, stream>>>(C, ldc, rows, cols, beta, tri);
  return cudaGetLastError();
}

}  // namespace sgb
