// Internal declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/strassen.h"

namespace sgb {

// Largest table the kernels take: 7^2 products with 2^2 terms per operand and up to
// 4 C targets (Eq. 3, Section 3.5).
constexpr int kMaxProducts = 49;
constexpr int kMaxTerms = 4;

// One term of a product: block (bi, bj) of the 2^L x 2^L partition with a sign.
// Encoded in one byte: bits 0-2 block column, bits 3-5 block row, bit 7 negative.
__host__ __device__ inline uint8_t term_code(int bi, int bj, int neg) {
  return (uint8_t)((bj & 7) | ((bi & 7) << 3) | (neg ? 0x80 : 0));
}
__host__ __device__ inline int term_bj(uint8_t c) { return c & 7; }
__host__ __device__ inline int term_bi(uint8_t c) { return (c >> 3) & 7; }
__host__ __device__ inline int term_neg(uint8_t c) { return (c >> 7) & 1; }

// The coefficient table of Eq. 4 for L levels, in the encoding above.
struct Plan {
  int levels = 0;
  int nprod = 0;
  uint8_t na[kMaxProducts], nb[kMaxProducts], nc[kMaxProducts];
  uint8_t ta[kMaxProducts][kMaxTerms], tb[kMaxProducts][kMaxTerms], tc[kMaxProducts][kMaxTerms];
};

// Builds the table for levels 0, 1 or 2 (Figure 1 and its Kronecker square).
// Returns false for other levels.
bool make_plan(int levels, Plan* out);

// Block edge h = ceil(d / 2^L) (Section 3.3, zero padding of the fringe).
inline int64_t block_edge(int64_t d, int levels) {
  const int64_t p = (int64_t)1 << levels;
  return (d + p - 1) / p;
}

// How partial products reach C (or the temporary M).
enum EpilogueKind : int {
  kEpiAtomicAdd = 0,  // red.global.add.f64 of +/- M into every target (any schedule)
  kEpiRmw = 1,        // load, add, store: only when one block owns the target tile
  kEpiStore = 2       // overwrite (AB / Naive temporary M): only when one block owns it
};

// How work units are spread over the persistent grid.
enum ScheduleKind : int {
  kSchedStreamK = 0,  // equal contiguous ranges of the (unit, k-step) space per block
  kSchedOwner = 1     // each block owns whole tile positions, all products, all of k
};

// One launch of the FP64 product kernel: all products of a plan over one (A, B, C).
struct Fp64Launch {
  const double* A;
  const double* B;
  double* C;
  int64_t lda, ldb, ldc;
  int64_t a_rows, a_cols;  // extent of A that holds data (m x k); beyond reads as zero
  int64_t b_rows, b_cols;  // extent of B (k x n)
  int64_t c_rows, c_cols;  // extent of C that may be written (m x n, or hm x hn for M)
  int64_t hm, hn, hk;      // block edges
  const Plan* plan;        // products to run (all of them, or one via `only_product`)
  int only_product;        // -1 = all products of the plan, else just this one
  EpilogueKind epi;
  ScheduleKind sched;
  int tile;                // tile configuration id (see fp64_gemm.cu)
};

// Launches the FP64 product kernel; returns a CUDA error code.
cudaError_t launch_fp64(const Fp64Launch& L, cudaStream_t stream);

// Number of tile configurations the FP64 kernel is built for.
int fp64_num_tiles();

// Picks a schedule and tile for a launch (balance heuristics for 152 SMs).
void choose_fp64_schedule(Fp64Launch* L, int prefer_deterministic);

// Naive / AB helpers (elementwise.cu).
// dst (rows x cols, ld = cols) = sum_t sign_t * block_t of src, masked to src's extent.
cudaError_t launch_block_sum(double* dst, int64_t rows, int64_t cols,
                             const double* src, int64_t ld, int64_t src_rows, int64_t src_cols,
                             int64_t h_r, int64_t h_c, const uint8_t* terms, int nterms,
                             cudaStream_t stream);
// For each target t: C block (bi, bj) += sign * M (hm x hn, ld = hn), masked to C.
cudaError_t launch_combine(double* C, int64_t ldc, int64_t c_rows, int64_t c_cols,
                           const double* M, int64_t hm, int64_t hn,
                           const uint8_t* targets, int ntargets, cudaStream_t stream);

int device_sm_count();

}  // namespace sgb
