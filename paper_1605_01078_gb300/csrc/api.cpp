// C ABI entry points (include/strassen.h): argument checks, plan selection and the
// launch sequences of the ABC, AB and Naive variants (Section 4.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "internal.h"

using namespace sgb;

namespace {

// Shared argument checks of strassen_gemm / classical_gemm.  Returns 1 when the call
// has nothing to do, 0 when it should proceed, or a negative status.
int check_args(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
               int64_t ldb, const double* C, int64_t ldc) {
  if (m < 0 || n < 0 || k < 0) return STRASSEN_ERR_DIM;
  if (m == 0 || n == 0 || k == 0) return 1;
  if (!A || !B || !C) return STRASSEN_ERR_NULL;
  if (lda < k || ldb < n || ldc < n) return STRASSEN_ERR_LD;
  // C must not overlap A or B (byte ranges of the three operands).
  const char* a0 = (const char*)A;
  const char* a1 = (const char*)(A + (m - 1) * lda + k);
  const char* b0 = (const char*)B;
  const char* b1 = (const char*)(B + (k - 1) * ldb + n);
  const char* c0 = (const char*)C;
  const char* c1 = (const char*)(C + (m - 1) * ldc + n);
  if ((c0 < a1 && a0 < c1) || (c0 < b1 && b0 < c1)) return STRASSEN_ERR_ARG;
  return 0;
}

// BLAS options of strassen_dgemm_ex: op(A), op(B), the scale of the product, and
// whether the rounding order must be the same on every run (STRASSEN_FLAG_DETERMINISTIC).
struct Op {
  int ta = 0, tb = 0;
  double alpha = 1.0;
  int det = 0;
};

// Argument checks of strassen_dgemm (stored shapes follow the transposes).  Returns 1
// when there is no product to compute, 0 when it should proceed, or a negative status.
int check_args_op(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                  int64_t ldb, const double* C, int64_t ldc, const Op& op) {
  if (m < 0 || n < 0 || k < 0) return STRASSEN_ERR_DIM;
  if (m == 0 || n == 0) return 1;
  if (!C) return STRASSEN_ERR_NULL;
  if (ldc < n) return STRASSEN_ERR_LD;
  if (k == 0 || op.alpha == 0.0) return 1;
  if (!A || !B) return STRASSEN_ERR_NULL;
  const int64_t ar = op.ta ? k : m, ac = op.ta ? m : k, br = op.tb ? n : k, bc = op.tb ? k : n;
  if (lda < ac || ldb < bc) return STRASSEN_ERR_LD;
  const char* a0 = (const char*)A;
  const char* a1 = (const char*)(A + (ar - 1) * lda + ac);
  const char* b0 = (const char*)B;
  const char* b1 = (const char*)(B + (br - 1) * ldb + bc);
  const char* c0 = (const char*)C;
  const char* c1 = (const char*)(C + (m - 1) * ldc + n);
  if ((c0 < a1 && a0 < c1) || (c0 < b1 && b0 < c1)) return STRASSEN_ERR_ARG;
  return 0;
}

int clamp_levels(int levels, int64_t m, int64_t n, int64_t k) {
  int64_t mn = m < n ? m : n;
  mn = mn < k ? mn : k;
  while (levels > 0 && ((int64_t)1 << levels) > mn) --levels;
  return levels;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? STRASSEN_OK : STRASSEN_ERR_CUDA; }

int run_classical(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                  int64_t ldb, double* C, int64_t ldc, EpilogueKind owner_epi, cudaStream_t s, int tile = -1,
                  const Op& op = Op()) {
  Fp64Launch L = make_launch(m, n, k, A, lda, B, ldb, C, ldc, 0);
  L.epi = owner_epi;
  L.tile = tile;
  L.trans_a = op.ta; L.trans_b = op.tb; L.alpha = op.alpha;
  choose_fp64_schedule(&L, op.det);
  if (owner_epi == kEpiStore) {
    // The kernel accumulates into its target: a store is a clear followed by the adds.
    if (cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * n, m, s) != cudaSuccess)
      return STRASSEN_ERR_CUDA;
  }
  return cuda_status(launch_fp64(L, s));
}

int run_abc(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
            int64_t ldb, double* C, int64_t ldc, int levels, cudaStream_t s, int tile, const Op& op = Op()) {
  Fp64Launch L = make_launch(m, n, k, A, lda, B, ldb, C, ldc, levels);
  L.epi = kEpiAtomicAdd;
  L.tile = tile;
  L.trans_a = op.ta; L.trans_b = op.tb; L.alpha = op.alpha;
  choose_fp64_schedule(&L, op.det);
  return cuda_status(launch_fp64(L, s));
}

struct Workspace {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  ~Workspace() {
    if (p) cudaFreeAsync(p, s);
  }
};

int run_ab(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
           int64_t ldb, double* C, int64_t ldc, int levels, cudaStream_t s, int tile, const Op& op = Op()) {
  Plan pl;
  if (!make_plan(levels, &pl)) return STRASSEN_ERR_LEVELS;
  const int64_t hm = block_edge(m, levels), hn = block_edge(n, levels);
  Workspace ws;
  ws.s = s;
  if (cudaMallocAsync(&ws.p, sizeof(double) * hm * hn, s) != cudaSuccess) {
    cudaGetLastError();
    ws.p = nullptr;
    return STRASSEN_ERR_ALLOC;
  }
  double* M = (double*)ws.p;
  for (int r = 0; r < pl.nprod; ++r) {
    // The product writes M_r (one target: block (0,0) of M, sign +) ...
    Fp64Launch L = make_launch(m, n, k, A, lda, B, ldb, M, hn, levels);
    L.c_rows = hm; L.c_cols = hn;
    L.prod_begin = r; L.nprod = 1;
    L.m_target = 1;
    L.epi = kEpiStore;
    L.tile = tile;
    L.trans_a = op.ta; L.trans_b = op.tb;  // alpha is applied by the C updates
    choose_fp64_schedule(&L, op.det);
    // The kernel accumulates into M: clear it first.
    if (cudaMemsetAsync(M, 0, sizeof(double) * hm * hn, s) != cudaSuccess) return STRASSEN_ERR_CUDA;
    cudaError_t e = launch_fp64(L, s);
    if (e != cudaSuccess) return STRASSEN_ERR_CUDA;
    // ... then the separate updates C_q += gamma_q alpha M_r.
    e = launch_combine(C, ldc, m, n, M, hm, hn, pl.tc[r], pl.nc[r], s, op.alpha);
    if (e != cudaSuccess) return STRASSEN_ERR_CUDA;
  }
  return STRASSEN_OK;
}

// Hybrid plan: AB at the outermost level, ABC below it.  For each outer product a the
// launch runs rows [7^(L-1) a, 7^(L-1) (a + 1)) of the L-level table (operand sums fused,
// as in ABC) and scatters them with the (L-1)-level table's coefficients into the
// temporary M_a (outer blocks of 2^(L-1) h); then M_a is added into C with the outer
// product's coefficients of Figure 1.
int run_hybrid(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
               double* C, int64_t ldc, int levels, cudaStream_t s, int tile, const Op& op = Op()) {
  if (levels < 2) return run_ab(m, n, k, A, lda, B, ldb, C, ldc, levels, s, tile, op);
  Plan outer;
  if (!make_plan(1, &outer)) return STRASSEN_ERR_LEVELS;
  const int64_t hm = block_edge(m, levels), hn = block_edge(n, levels);
  const int64_t sub = (int64_t)1 << (levels - 1);
  const int64_t om = sub * hm, on = sub * hn;  // the outer blocks of the L-level partition
  Workspace ws;
  ws.s = s;
  if (cudaMallocAsync(&ws.p, sizeof(double) * om * on, s) != cudaSuccess) {
    cudaGetLastError();
    ws.p = nullptr;
    return STRASSEN_ERR_ALLOC;
  }
  double* M = (double*)ws.p;
  const int inner = kPlanCount[levels - 1];
  for (int a = 0; a < 7; ++a) {
    Fp64Launch L = make_launch(m, n, k, A, lda, B, ldb, M, on, levels);
    L.c_rows = om; L.c_cols = on;
    L.prod_begin = a * inner; L.nprod = inner;
    L.inner_targets = 1;
    L.epi = kEpiStore;
    L.tile = tile;
    L.trans_a = op.ta; L.trans_b = op.tb;  // alpha is applied by the C updates
    choose_fp64_schedule(&L, op.det);
    if (cudaMemsetAsync(M, 0, sizeof(double) * om * on, s) != cudaSuccess) return STRASSEN_ERR_CUDA;
    if (launch_fp64(L, s) != cudaSuccess) return STRASSEN_ERR_CUDA;
    if (launch_combine(C, ldc, m, n, M, om, on, outer.tc[a], outer.nc[a], s, op.alpha) != cudaSuccess)
      return STRASSEN_ERR_CUDA;
  }
  return STRASSEN_OK;
}

int run_naive(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
              int64_t ldb, double* C, int64_t ldc, int levels, cudaStream_t s, int tile, const Op& op = Op()) {
  Plan pl;
  if (!make_plan(levels, &pl)) return STRASSEN_ERR_LEVELS;
  const int64_t hm = block_edge(m, levels), hn = block_edge(n, levels), hk = block_edge(k, levels);
  Workspace ws;
  ws.s = s;
  const int64_t elems = hm * hk + hk * hn + hm * hn;
  if (cudaMallocAsync(&ws.p, sizeof(double) * elems, s) != cudaSuccess) {
    cudaGetLastError();
    ws.p = nullptr;
    return STRASSEN_ERR_ALLOC;
  }
  double* X = (double*)ws.p;
  double* V = X + hm * hk;
  double* M = V + hk * hn;
  for (int r = 0; r < pl.nprod; ++r) {
    cudaError_t e = launch_block_sum(X, hm, hk, A, lda, m, k, hm, hk, pl.ta[r], pl.na[r], s, op.ta);
    if (e != cudaSuccess) return STRASSEN_ERR_CUDA;
    e = launch_block_sum(V, hk, hn, B, ldb, k, n, hk, hn, pl.tb[r], pl.nb[r], s, op.tb);
    if (e != cudaSuccess) return STRASSEN_ERR_CUDA;
    Op inner;
    inner.det = op.det;
    int st = run_classical(hm, hn, hk, X, hk, V, hn, M, hn, kEpiStore, s, tile, inner);
    if (st != STRASSEN_OK) return st;
    e = launch_combine(C, ldc, m, n, M, hm, hn, pl.tc[r], pl.nc[r], s, op.alpha);
    if (e != cudaSuccess) return STRASSEN_ERR_CUDA;
  }
  return STRASSEN_OK;
}

int run_oz(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
           double* C, int64_t ldc, int levels, cudaStream_t s, const Op& op = Op()) {
  Workspace ws;
  ws.s = s;
  if (cudaMallocAsync(&ws.p, (size_t)ozaki_workspace_bytes(m, n, k, levels), s) != cudaSuccess) {
    cudaGetLastError();
    ws.p = nullptr;
    return STRASSEN_ERR_ALLOC;
  }
  return cuda_status(run_ozaki(m, n, k, A, lda, B, ldb, C, ldc, levels, ws.p, s, op.ta, op.tb, op.alpha));
}

// A non-blocking library stream per device for the second branch of a batched call.
cudaError_t side_stream(cudaStream_t* out) {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!streams[dev]) {
    e = cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  *out = streams[dev];
  return cudaSuccess;
}

// The selection of strassen_select (exhaustive record, then the learned selector, then
// the analytic model or, for split precision, classical slices).  With may_launch = 0
// the learned selector answers only from its cache of earlier choices (no kernel launch
// and no wait), as inside a stream capture.
void select_plan(int64_t m, int64_t n, int64_t k, int dtype, int may_launch, int* levels, strassen_variant* variant,
                 int* tile_id) {
  int lv = 0, var = STRASSEN_ABC, tile = 0, cand = -1;
  if (record_lookup(m, n, k, dtype, &lv, &var, &tile)) {
    // exhaustive measurement
  } else if (m > 0 && n > 0 && k > 0 && mlp_select(m, n, k, dtype, may_launch, &cand)) {
    selector_candidate(cand, &lv, &var, &tile);
  } else if (dtype == STRASSEN_F64) {
    model_select(m, n, k, &lv, &var, &tile);
  } else {  // split precision: classical slices
    lv = 0;
    var = STRASSEN_ABC;
    tile = 0;
  }
  *levels = lv;
  *variant = (strassen_variant)var;
  *tile_id = tile;
}

// The product C += alpha op(A) op(B) with the requested (or selected) plan; arguments
// already checked.
int run_product(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
                double* C, int64_t ldc, int levels, strassen_variant variant, strassen_dtype dtype, cudaStream_t s,
                const Op& op) {
  if (dtype == STRASSEN_F64_OZ_INT8) return STRASSEN_ERR_UNSUPPORTED;
  int tile = -1;  // the launch's own choice unless the selector picked the whole plan
  if (levels == -1 || variant == STRASSEN_AUTO) {
    int sl = 0, st_tile = 0;
    strassen_variant sv = STRASSEN_ABC;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
      cudaGetLastError();
      cap = cudaStreamCaptureStatusActive;
    }
    select_plan(m, n, k, (int)dtype, cap == cudaStreamCaptureStatusNone, &sl, &sv, &st_tile);
    if (levels == -1 && variant == STRASSEN_AUTO) tile = st_tile;
    if (levels == -1) levels = sl;
    if (variant == STRASSEN_AUTO) variant = sv;
  }
  const int requested_levels = levels;
  levels = clamp_levels(levels, m, n, k);
  if (levels != requested_levels) tile = -1;
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return STRASSEN_ERR_CUDA;
  }
  if (dtype == STRASSEN_F64_OZ_BF16) return run_oz(m, n, k, A, lda, B, ldb, C, ldc, levels, s, op);
  if (levels == 0) return run_classical(m, n, k, A, lda, B, ldb, C, ldc, kEpiRmw, s, tile, op);
  switch (variant) {
    case STRASSEN_ABC: return run_abc(m, n, k, A, lda, B, ldb, C, ldc, levels, s, tile, op);
    case STRASSEN_AB: return run_ab(m, n, k, A, lda, B, ldb, C, ldc, levels, s, tile, op);
    case STRASSEN_NAIVE: return run_naive(m, n, k, A, lda, B, ldb, C, ldc, levels, s, tile, op);
    case STRASSEN_HYBRID: return run_hybrid(m, n, k, A, lda, B, ldb, C, ldc, levels, s, tile, op);
    default: return STRASSEN_ERR_UNSUPPORTED;
  }
}

// Symmetric rank-k update, recursively: the diagonal blocks by the same recursion
// down to kSyrkLeaf rows, where one classical launch writes only the triangle; the
// off-diagonal block by the Strassen product with the transposed operand read in place.
constexpr int64_t kSyrkLeaf = 1024;

int run_syrk(int uplo, int trans, int64_t n, int64_t k, double alpha, const double* A, int64_t lda, double* C,
             int64_t ldc, int levels, cudaStream_t s, int det) {
  if (n <= 0) return STRASSEN_OK;
  // Row r of op(A) (k long): A + r * lda for trans = 0, column r of A (A + r) for trans = 1.
  auto row_block = [&](int64_t r0) { return trans ? A + r0 : A + r0 * lda; };
  if (n <= kSyrkLeaf) {
    Fp64Launch L = make_launch(n, n, k, A, lda, A, lda, C, ldc, 0);
    L.trans_a = trans;       // op(A)
    L.trans_b = 1 - trans;   // op(A)^T: the same storage read the other way
    L.alpha = alpha;
    L.tri = uplo == 0 ? 1 : 2;
    L.epi = kEpiRmw;
    choose_fp64_schedule(&L, det);
    return cuda_status(launch_fp64(L, s));
  }
  // Split near the middle, on a multiple of 128 rows where one lies inside.
  int64_t n0 = (n + 1) / 2;
  if (n0 > 128) n0 = n0 / 128 * 128;
  int st = run_syrk(uplo, trans, n0, k, alpha, A, lda, C, ldc, levels, s, det);
  if (st != STRASSEN_OK) return st;
  const int64_t n1 = n - n0;
  st = run_syrk(uplo, trans, n1, k, alpha, row_block(n0), lda, C + n0 * ldc + n0, ldc, levels, s, det);
  if (st != STRASSEN_OK) return st;
  Op op;
  op.alpha = alpha;
  op.det = det;
  // lower: C10 (n1 x n0) += alpha op(A)_1 op(A)_0^T; upper: C01 (n0 x n1) += alpha op(A)_0 op(A)_1^T
  const double* Ar = uplo == 0 ? row_block(n0) : row_block(0);
  const double* Ac = uplo == 0 ? row_block(0) : row_block(n0);
  const int64_t mr = uplo == 0 ? n1 : n0, nc = uplo == 0 ? n0 : n1;
  double* Cb = uplo == 0 ? C + n0 * ldc : C + n0;
  op.ta = trans;
  op.tb = 1 - trans;
  const strassen_variant v = levels == -1 ? STRASSEN_AUTO : STRASSEN_ABC;
  return run_product(mr, nc, k, Ar, lda, Ac, lda, Cb, ldc, levels, v, STRASSEN_F64, s, op);
}

}  // namespace

extern "C" {

int strassen_dsyrk(int uplo, int trans, int64_t n, int64_t k, double alpha, const double* A, int64_t lda, double beta,
                   double* C, int64_t ldc, int levels, unsigned flags, strassen_stream_t stream) {
  try {
    if (uplo < 0 || uplo > 1 || trans < 0 || trans > 1) return STRASSEN_ERR_ARG;
    if (flags & ~(unsigned)STRASSEN_FLAG_DETERMINISTIC) return STRASSEN_ERR_ARG;
    if (levels < -1 || levels > kMaxLevels) return STRASSEN_ERR_LEVELS;
    if (n < 0 || k < 0) return STRASSEN_ERR_DIM;
    if (n == 0) return STRASSEN_OK;
    if (!C) return STRASSEN_ERR_NULL;
    if (ldc < n) return STRASSEN_ERR_LD;
    const bool product = k > 0 && alpha != 0.0;
    if (product) {
      if (!A) return STRASSEN_ERR_NULL;
      const int64_t ar = trans ? k : n, ac = trans ? n : k;
      if (lda < ac) return STRASSEN_ERR_LD;
      const char* a0 = (const char*)A;
      const char* a1 = (const char*)(A + (ar - 1) * lda + ac);
      const char* c0 = (const char*)C;
      const char* c1 = (const char*)(C + (n - 1) * ldc + n);
      if (c0 < a1 && a0 < c1) return STRASSEN_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaPeekAtLastError() != cudaSuccess) {
      cudaGetLastError();
      return STRASSEN_ERR_CUDA;
    }
    // C = beta C on the triangle (beta = 0 writes zeros), then the products with beta 1.
    if (launch_scale(C, ldc, n, n, beta, s, uplo == 0 ? 1 : 2) != cudaSuccess) return STRASSEN_ERR_CUDA;
    if (!product) return STRASSEN_OK;
    return run_syrk(uplo, trans, n, k, alpha, A, lda, C, ldc, levels, s, (flags & STRASSEN_FLAG_DETERMINISTIC) ? 1 : 0);
  } catch (...) {
    return STRASSEN_ERR_ALLOC;
  }
}


int strassen_gemm(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                  int64_t ldb, double* C, int64_t ldc, int levels, strassen_variant variant,
                  strassen_dtype dtype, strassen_stream_t stream) {
  try {
    if (levels < -1 || levels > kMaxLevels) return STRASSEN_ERR_LEVELS;
    if ((int)variant < 0 || (int)variant > 4) return STRASSEN_ERR_UNSUPPORTED;
    if ((int)dtype < 0 || (int)dtype > 2) return STRASSEN_ERR_UNSUPPORTED;
    const int chk = check_args(m, n, k, A, lda, B, ldb, C, ldc);
    if (chk < 0) return chk;
    if (chk == 1) return STRASSEN_OK;
    return run_product(m, n, k, A, lda, B, ldb, C, ldc, levels, variant, dtype, (cudaStream_t)stream, Op());
  } catch (...) {
    return STRASSEN_ERR_ALLOC;
  }
}

int strassen_dgemm_ex(int transa, int transb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                      int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int levels,
                      strassen_variant variant, strassen_dtype dtype, unsigned flags, strassen_stream_t stream) {
  try {
    if (transa < 0 || transa > 1 || transb < 0 || transb > 1) return STRASSEN_ERR_ARG;
    if (flags & ~(unsigned)STRASSEN_FLAG_DETERMINISTIC) return STRASSEN_ERR_ARG;
    if (levels < -1 || levels > kMaxLevels) return STRASSEN_ERR_LEVELS;
    if ((int)variant < 0 || (int)variant > 4) return STRASSEN_ERR_UNSUPPORTED;
    if ((int)dtype < 0 || (int)dtype > 2) return STRASSEN_ERR_UNSUPPORTED;
    Op op;
    op.ta = transa; op.tb = transb; op.alpha = alpha;
    op.det = (flags & STRASSEN_FLAG_DETERMINISTIC) ? 1 : 0;
    const int chk = check_args_op(m, n, k, A, lda, B, ldb, C, ldc, op);
    if (chk < 0) return chk;
    if (m == 0 || n == 0) return STRASSEN_OK;
    if (dtype == STRASSEN_F64_OZ_INT8) return STRASSEN_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    // C = beta C first (BLAS: beta = 0 ignores what C held), then C += alpha op(A) op(B).
    if (launch_scale(C, ldc, m, n, beta, s) != cudaSuccess) return STRASSEN_ERR_CUDA;
    if (chk == 1) return STRASSEN_OK;
    return run_product(m, n, k, A, lda, B, ldb, C, ldc, levels, variant, dtype, s, op);
  } catch (...) {
    return STRASSEN_ERR_ALLOC;
  }
}

int strassen_dgemm(int transa, int transb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                   int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int levels,
                   strassen_variant variant, strassen_dtype dtype, strassen_stream_t stream) {
  return strassen_dgemm_ex(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, levels, variant, dtype, 0u,
                           stream);
}

int classical_gemm(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                   int64_t ldb, double* C, int64_t ldc, strassen_stream_t stream) {
  try {
    const int chk = check_args(m, n, k, A, lda, B, ldb, C, ldc);
    if (chk < 0) return chk;
    if (chk == 1) return STRASSEN_OK;
    if (cudaPeekAtLastError() != cudaSuccess) {
      cudaGetLastError();
      return STRASSEN_ERR_CUDA;
    }
    return run_classical(m, n, k, A, lda, B, ldb, C, ldc, kEpiRmw, (cudaStream_t)stream);
  } catch (...) {
    return STRASSEN_ERR_ALLOC;
  }
}

int strassen_gemm_batched(int count, const strassen_problem* probs, strassen_dtype dtype,
                          strassen_stream_t stream) {
  try {
    if (count < 0) return STRASSEN_ERR_ARG;
    if (count == 0) return STRASSEN_OK;
    if (!probs) return STRASSEN_ERR_NULL;
    if ((int)dtype < 0 || (int)dtype > 2) return STRASSEN_ERR_UNSUPPORTED;
    if (dtype != STRASSEN_F64) return STRASSEN_ERR_UNSUPPORTED;
    std::vector<Fp64Launch> launches;
    std::vector<char> free_levels;  // 1: the level is chosen below, jointly with the tile
    std::vector<std::pair<const char*, const char*>> cranges;
    launches.reserve(count);
    for (int i = 0; i < count; ++i) {
      const strassen_problem& p = probs[i];
      if (p.levels < -1 || p.levels > kMaxLevels) return STRASSEN_ERR_LEVELS;
      if ((int)p.variant < 0 || (int)p.variant > 4) return STRASSEN_ERR_UNSUPPORTED;
      // The persistent launch runs the fused (ABC) form only: AB, Naive and the hybrid
      // plan need their temporaries and separate passes per product.
      if ((p.variant == STRASSEN_AB || p.variant == STRASSEN_NAIVE || p.variant == STRASSEN_HYBRID) &&
          p.levels != 0)
        return STRASSEN_ERR_UNSUPPORTED;
      const int chk = check_args(p.m, p.n, p.k, p.A, p.lda, p.B, p.ldb, p.C, p.ldc);
      if (chk < 0) return chk;
      if (chk == 1) continue;
      int levels = p.levels;
      bool chosen_here = false;
      if (levels == -1) {
        int rl = 0, rv = 0, rt = 0;
        if (record_lookup(p.m, p.n, p.k, (int)dtype, &rl, &rv, &rt)) levels = rl;  // exhaustive record
        else chosen_here = true;
      }
      levels = chosen_here ? 0 : clamp_levels(levels, p.m, p.n, p.k);
      launches.push_back(make_launch(p.m, p.n, p.k, p.A, p.lda, p.B, p.ldb, p.C, p.ldc, levels));
      free_levels.push_back(chosen_here ? 1 : 0);
      cranges.emplace_back((const char*)p.C, (const char*)(p.C + (p.m - 1) * p.ldc + p.n));
    }
    if (launches.empty()) return STRASSEN_OK;
    // Each problem takes the block tile (and, when free, the level) with the smallest
    // estimate of its padded tile work; the problems of one tile share one persistent
    // launch, so the call makes one launch per tile in use (at most two).
    for (size_t i = 0; i < launches.size(); ++i) {
      const Fp64Launch L = launches[i];
      const int64_t m = L.a_rows, k = L.a_cols, n = L.b_cols;
      const int lv_hi = free_levels[i] ? clamp_levels(kMaxLevels, m, n, k) : L.levels;
      const int lv_lo = free_levels[i] ? 0 : L.levels;
      double b = 1e300;
      int bl = L.levels, bt = 0;
      for (int lv = lv_lo; lv <= lv_hi; ++lv) {
        const Fp64Launch Lv = make_launch(m, n, k, L.A, L.lda, L.B, L.ldb, L.C, L.ldc, lv);
        for (int t = 0; t < kNumTiles; ++t) {
          const double x = fp64_launch_estimate(Lv, t, 1);
          if (x < b * 0.99) { b = x; bl = lv; bt = t; }  // fewer levels, then the larger tile, within 1 %
        }
      }
      launches[i] = make_launch(m, n, k, L.A, L.lda, L.B, L.ldb, L.C, L.ldc, bl);
      launches[i].tile = bt;
    }
    // The C ranges of different problems must not overlap (atomics would mix them).
    std::sort(cranges.begin(), cranges.end());
    for (size_t i = 1; i < cranges.size(); ++i)
      if (cranges[i].first < cranges[i - 1].second) return STRASSEN_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaPeekAtLastError() != cudaSuccess) {
      cudaGetLastError();
      return STRASSEN_ERR_CUDA;
    }
    // One persistent launch per block tile in use, the larger first, the second on a
    // library stream forked from the caller's, so that the first launch's tail overlaps
    // the second's start; the caller's stream waits for both at the end.
    std::stable_sort(launches.begin(), launches.end(),
                     [](const Fp64Launch& a, const Fp64Launch& b) { return a.tile < b.tile; });
    struct Group {
      size_t begin, end;
      double work;
    };
    std::vector<Group> groups;
    size_t scratch_bytes = 0;
    for (size_t i = 0; i < launches.size();) {
      size_t j = i;
      double w = 0.0;
      while (j < launches.size() && launches[j].tile == launches[i].tile) {
        w += fp64_launch_estimate(launches[j], launches[j].tile, 1);
        ++j;
      }
      groups.push_back(Group{i, j, w});
      scratch_bytes += (fp64_batched_scratch_bytes((int)(j - i)) + 255) / 256 * 256;
      i = j;
    }
    std::stable_sort(groups.begin(), groups.end(), [](const Group& a, const Group& b) { return a.work > b.work; });
    Workspace ws;
    ws.s = s;
    if (cudaMallocAsync(&ws.p, scratch_bytes, s) != cudaSuccess) {
      cudaGetLastError();
      ws.p = nullptr;
      return STRASSEN_ERR_ALLOC;
    }
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    if (groups.size() > 1) {
      if (side_stream(&side) != cudaSuccess || cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventRecord(fork, s) != cudaSuccess || cudaStreamWaitEvent(side, fork, 0) != cudaSuccess) {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        return STRASSEN_ERR_CUDA;
      }
    }
    int st = STRASSEN_OK;
    char* scratch = (char*)ws.p;
    for (size_t g = 0; g < groups.size() && st == STRASSEN_OK; ++g) {
      const int cnt = (int)(groups[g].end - groups[g].begin);
      cudaStream_t gs = (g % 2 == 0) ? s : side;
      if (launch_fp64_batched(launches.data() + groups[g].begin, cnt, scratch, gs) != cudaSuccess)
        st = STRASSEN_ERR_CUDA;
      scratch += (fp64_batched_scratch_bytes(cnt) + 255) / 256 * 256;
    }
    if (side) {
      if (cudaEventRecord(join, side) != cudaSuccess || cudaStreamWaitEvent(s, join, 0) != cudaSuccess)
        st = STRASSEN_ERR_CUDA;
      cudaEventDestroy(fork);
      cudaEventDestroy(join);
    }
    return st;
  } catch (...) {
    return STRASSEN_ERR_ALLOC;
  }
}

int strassen_device_status(strassen_stream_t stream) {
  const int a = fp64_device_status((cudaStream_t)stream);
  const int b = ozaki_device_status();
  return a != STRASSEN_OK ? a : b;
}

int strassen_check_int_fadd(int64_t count, uint64_t seed, uint64_t* mismatches, strassen_stream_t stream) {
  if (count < 0) return STRASSEN_ERR_ARG;
  if (!mismatches) return STRASSEN_ERR_NULL;
  unsigned long long mm = 0;
  const cudaError_t e = check_int_fadd((long long)count, (unsigned long long)seed, &mm, (cudaStream_t)stream);
  if (e != cudaSuccess) return STRASSEN_ERR_CUDA;
  *mismatches = (uint64_t)mm;
  return STRASSEN_OK;
}

int strassen_profile_split_precision(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                                     int64_t ldb, double* C, int64_t ldc, int levels, float* stage_ms,
                                     strassen_stream_t stream) {
  try {
    if (!stage_ms) return STRASSEN_ERR_NULL;
    if (levels < 0 || levels > kMaxLevels) return STRASSEN_ERR_LEVELS;
    const int chk = check_args(m, n, k, A, lda, B, ldb, C, ldc);
    if (chk < 0) return chk;
    stage_ms[0] = stage_ms[1] = stage_ms[2] = 0.0f;
    if (chk == 1) return STRASSEN_OK;
    levels = clamp_levels(levels, m, n, k);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int st = STRASSEN_OK;
    for (int i = 0; i < 4 && st == STRASSEN_OK; ++i)
      if (cudaEventCreate(&ev[i]) != cudaSuccess) st = STRASSEN_ERR_CUDA;
    if (st == STRASSEN_OK) {
      Workspace ws;
      ws.s = s;
      if (cudaMallocAsync(&ws.p, (size_t)ozaki_workspace_bytes(m, n, k, levels), s) != cudaSuccess) {
        cudaGetLastError();
        ws.p = nullptr;
        st = STRASSEN_ERR_ALLOC;
      } else {
        st = cuda_status(run_ozaki(m, n, k, A, lda, B, ldb, C, ldc, levels, ws.p, s, 0, 0, 1.0, ev));
      }
    }
    if (st == STRASSEN_OK && cudaEventSynchronize(ev[3]) != cudaSuccess) st = STRASSEN_ERR_CUDA;
    for (int i = 0; i < 3 && st == STRASSEN_OK; ++i)
      if (cudaEventElapsedTime(&stage_ms[i], ev[i], ev[i + 1]) != cudaSuccess) st = STRASSEN_ERR_CUDA;
    for (int i = 0; i < 4; ++i)
      if (ev[i]) cudaEventDestroy(ev[i]);
    return st;
  } catch (...) {
    return STRASSEN_ERR_ALLOC;
  }
}

int strassen_check_wait_timeout(int64_t limit_cycles, strassen_stream_t stream) {
  if (limit_cycles < 0) return STRASSEN_ERR_ARG;
  return cuda_status(launch_wait_timeout_check((long long)limit_cycles, (cudaStream_t)stream));
}

int strassen_select(int64_t m, int64_t n, int64_t k, strassen_dtype dtype, int* levels,
                    strassen_variant* variant, int* tile_id) {
  if (!levels || !variant || !tile_id) return STRASSEN_ERR_NULL;
  if (m < 0 || n < 0 || k < 0) return STRASSEN_ERR_DIM;
  if ((int)dtype < 0 || (int)dtype > 2) return STRASSEN_ERR_UNSUPPORTED;
  try {
    select_plan(m, n, k, (int)dtype, 1, levels, variant, tile_id);
  } catch (...) {
    return STRASSEN_ERR_ALLOC;
  }
  return STRASSEN_OK;
}

int strassen_tune_record(int64_t m, int64_t n, int64_t k, strassen_dtype dtype, int levels,
                         strassen_variant variant, int tile_id) {
  if (m < 0 || n < 0 || k < 0) return STRASSEN_ERR_DIM;
  if (levels < 0 || levels > kMaxLevels) return STRASSEN_ERR_LEVELS;
  if ((int)dtype < 0 || (int)dtype > 2 || (int)variant < 0 || (int)variant > 2) return STRASSEN_ERR_UNSUPPORTED;
  if (tile_id < 0 || tile_id >= kNumTiles) return STRASSEN_ERR_ARG;
  record_store(m, n, k, (int)dtype, levels, (int)variant, tile_id);
  return STRASSEN_OK;
}

int strassen_tune_clear(void) {
  record_clear();
  return STRASSEN_OK;
}

double strassen_model_seconds(int64_t m, int64_t n, int64_t k, int levels, strassen_variant variant) {
  if (m <= 0 || n <= 0 || k <= 0 || levels < 0 || levels > kMaxLevels || (int)variant < 0 || (int)variant > 2) return -1.0;
  double best = 1e300;
  for (int t = 0; t < kNumTiles; ++t) best = std::min(best, model_seconds(m, n, k, levels, (int)variant, t));
  return best;
}

int64_t strassen_workspace_size(int64_t m, int64_t n, int64_t k, int levels, strassen_variant variant,
                                strassen_dtype dtype) {
  if (m < 0 || n < 0 || k < 0) return STRASSEN_ERR_DIM;
  if (levels < -1 || levels > kMaxLevels) return STRASSEN_ERR_LEVELS;
  if ((int)variant < 0 || (int)variant > 4 || (int)dtype < 0 || (int)dtype > 2)
    return STRASSEN_ERR_UNSUPPORTED;
  if (m == 0 || n == 0 || k == 0) return 0;
  if (levels == -1 || variant == STRASSEN_AUTO) {
    int sl = 0, sel_tile = 0;
    strassen_variant sv = STRASSEN_ABC;
    strassen_select(m, n, k, dtype, &sl, &sv, &sel_tile);
    if (levels == -1) levels = sl;
    if (variant == STRASSEN_AUTO) variant = sv;
  }
  levels = clamp_levels(levels, m, n, k);
  if (dtype == STRASSEN_F64_OZ_INT8) return STRASSEN_ERR_UNSUPPORTED;
  if (dtype == STRASSEN_F64_OZ_BF16) return ozaki_workspace_bytes(m, n, k, levels);
  if (levels == 0 || variant == STRASSEN_ABC) return 0;
  const int64_t hm = block_edge(m, levels), hn = block_edge(n, levels), hk = block_edge(k, levels);
  if (variant == STRASSEN_AB || (variant == STRASSEN_HYBRID && levels < 2)) return (int64_t)sizeof(double) * hm * hn;
  if (variant == STRASSEN_HYBRID) {
    const int64_t sub = (int64_t)1 << (levels - 1);
    return (int64_t)sizeof(double) * (sub * hm) * (sub * hn);
  }
  return (int64_t)sizeof(double) * (hm * hk + hk * hn + hm * hn);
}

const char* strassen_status_string(int status) {
  switch (status) {
    case STRASSEN_OK: return "ok";
    case STRASSEN_ERR_DIM: return "negative dimension";
    case STRASSEN_ERR_LD: return "leading dimension smaller than the row length";
    case STRASSEN_ERR_NULL: return "null pointer for a non-empty operand";
    case STRASSEN_ERR_LEVELS: return "unsupported number of Strassen levels";
    case STRASSEN_ERR_UNSUPPORTED: return "unsupported dtype or variant";
    case STRASSEN_ERR_CUDA: return "CUDA error";
    case STRASSEN_ERR_TIMEOUT: return "device-side wait timed out";
    case STRASSEN_ERR_ALLOC: return "allocation failed";
    case STRASSEN_ERR_ARG: return "invalid argument";
    case STRASSEN_ERR_SCRATCH_LIMIT: return "product too large for the fixed scratch array of the no-allocation entry point";
    default: return "unknown status";
  }
}

int strassen_plan_table(int levels, int capacity, int* na, int* nb, int* nc, int* a_terms,
                        int* b_terms, int* c_terms) {
  Plan pl;
  if (!make_plan(levels, &pl)) return STRASSEN_ERR_LEVELS;
  if (!na || !nb || !nc || !a_terms || !b_terms || !c_terms) return STRASSEN_ERR_NULL;
  if (capacity < pl.nprod) return STRASSEN_ERR_ARG;
  auto enc = [](uint8_t c) { return (term_bi(c) * 16 + term_bj(c)) * 2 + term_neg(c); };
  for (int r = 0; r < pl.nprod; ++r) {
    na[r] = pl.na[r]; nb[r] = pl.nb[r]; nc[r] = pl.nc[r];
    for (int t = 0; t < kMaxTerms; ++t) {
      a_terms[r * kMaxTerms + t] = t < pl.na[r] ? enc(pl.ta[r][t]) : -1;
      b_terms[r * kMaxTerms + t] = t < pl.nb[r] ? enc(pl.tb[r][t]) : -1;
      c_terms[r * kMaxTerms + t] = t < pl.nc[r] ? enc(pl.tc[r][t]) : -1;
    }
  }
  return pl.nprod;
}

}  // extern "C"
