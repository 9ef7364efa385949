// strassen_gemm_ab_noalloc: the AB variant with its temporary M held in a fixed,
// library-owned device array instead of memory allocated per call.
//
// Who needs this: callers that must not allocate device memory while they run --
// a process whose device memory is already claimed by its own pooling allocator (so a
// cudaMalloc/cudaMallocAsync from inside the library can fail or fragment that pool),
// latency-bound loops where an allocation or a free may synchronise the device, and
// code that must not have a failure path for "out of memory" in the middle of its
// work.  The price: the array (kNoAllocMaxElems doubles, 32 MiB) is reserved on every
// GPU that loads the library until the process exits, and calls share it.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace sgb {
namespace {

// 4 Mi doubles = 32 MiB: room for M of (m/2^L) x (n/2^L) <= 2048 x 2048.
constexpr int64_t kNoAllocMaxElems = (int64_t)1 << 22;

static __device__ __align__(256) double g_ab_scratch[kNoAllocMaxElems];

// Device address of g_ab_scratch per device (the host-side symbol is only a stand-in
// and must never be passed to a kernel).
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_ab_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = (double*)g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace sgb

using namespace sgb;

namespace {

int ab_noalloc(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
               double* C, int64_t ldc, int levels, strassen_stream_t stream) {
  if (levels < 1 || levels > kMaxLevels) return STRASSEN_ERR_LEVELS;
  if (m < 0 || n < 0 || k < 0) return STRASSEN_ERR_DIM;
  if (m == 0 || n == 0 || k == 0) return STRASSEN_OK;
  if (!A || !B || !C) return STRASSEN_ERR_NULL;
  if (lda < k || ldb < n || ldc < n) return STRASSEN_ERR_LD;
  {
    const char* a0 = (const char*)A;
    const char* a1 = (const char*)(A + (m - 1) * lda + k);
    const char* b0 = (const char*)B;
    const char* b1 = (const char*)(B + (k - 1) * ldb + n);
    const char* c0 = (const char*)C;
    const char* c1 = (const char*)(C + (m - 1) * ldc + n);
    if ((c0 < a1 && a0 < c1) || (c0 < b1 && b0 < c1)) return STRASSEN_ERR_ARG;
  }
  int64_t mn = m < n ? m : n;
  mn = mn < k ? mn : k;
  while (levels > 0 && ((int64_t)1 << levels) > mn) --levels;
  if (levels == 0) return classical_gemm(m, n, k, A, lda, B, ldb, C, ldc, stream);
  const int64_t hm = block_edge(m, levels), hn = block_edge(n, levels);
  if (hm * hn > kNoAllocMaxElems) return STRASSEN_ERR_SCRATCH_LIMIT;

  cudaStream_t s = (cudaStream_t)stream;
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return STRASSEN_ERR_CUDA;
  }
  double* M = nullptr;
  if (scratch_address(&M) != cudaSuccess) {
    cudaGetLastError();
    return STRASSEN_ERR_CUDA;
  }
  Plan pl;
  if (!make_plan(levels, &pl)) return STRASSEN_ERR_LEVELS;
  for (int r = 0; r < pl.nprod; ++r) {
    // Each product writes M_r into block (0,0) of M with sign +.
    Fp64Launch L = make_launch(m, n, k, A, lda, B, ldb, M, hn, levels);
    L.c_rows = hm; L.c_cols = hn;
    L.prod_begin = r; L.nprod = 1;
    L.m_target = 1;
    L.epi = kEpiStore;
    choose_fp64_schedule(&L, 0);
    // The array keeps the previous call's contents and the kernel accumulates into
    // it: clear M first.
    if (cudaMemsetAsync(M, 0, sizeof(double) * hm * hn, s) != cudaSuccess) return STRASSEN_ERR_CUDA;
    if (launch_fp64(L, s) != cudaSuccess) return STRASSEN_ERR_CUDA;
    if (launch_combine(C, ldc, m, n, M, hm, hn, pl.tc[r], pl.nc[r], s) != cudaSuccess)
      return STRASSEN_ERR_CUDA;
  }
  return STRASSEN_OK;
}

}  // namespace

extern "C" int strassen_gemm_ab_noalloc(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                                        const double* B, int64_t ldb, double* C, int64_t ldc, int levels,
                                        strassen_stream_t stream) {
  // No exception may leave a C entry point (the set-up takes a lock, which can throw).
  try {
    return ab_noalloc(m, n, k, A, lda, B, ldb, C, ldc, levels, stream);
  } catch (...) {
    return STRASSEN_ERR_CUDA;
  }
}
