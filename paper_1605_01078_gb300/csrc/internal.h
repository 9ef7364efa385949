// Internal declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/strassen.h"
#include "plan_tables.h"

namespace sgb {

constexpr int kMaxProducts = 343;

// Host copy of the table of one level count (rows of kPlanTables).
struct Plan {
  int levels = 0;
  int nprod = 0;
  uint8_t na[kMaxProducts], nb[kMaxProducts], nc[kMaxProducts];
  uint8_t ta[kMaxProducts][kMaxTerms], tb[kMaxProducts][kMaxTerms], tc[kMaxProducts][kMaxTerms];
};

// Copies the table for levels 0..kMaxLevels (Figure 1 and its Kronecker powers).
// Returns false for other levels.
bool make_plan(int levels, Plan* out);

// Block edge h = ceil(d / 2^L) (Section 3.3, zero padding of the fringe).
inline int64_t block_edge(int64_t d, int levels) {
  const int64_t p = (int64_t)1 << levels;
  return (d + p - 1) / p;
}

// What the caller wants done with a product: accumulate into C, or store into a
// temporary (the kernel always accumulates with device atomics; a store is a clear of
// the target followed by the adds).
enum EpilogueKind : int {
  kEpiAtomicAdd = 0,  // accumulate, any schedule
  kEpiRmw = 1,        // accumulate with one owner per tile (deterministic order)
  kEpiStore = 2       // the target is a temporary that the caller clears first
};

// How work units are spread over the persistent grid.
enum ScheduleKind : int {
  kSchedStreamK = 0,  // equal contiguous ranges of the (unit, k-step) space per block
  kSchedOwner = 1     // each block owns whole tile positions, all products, all of k
};

// One problem for the FP64 product kernel: products [prod_begin, prod_begin + nprod)
// of the `levels` table over (A, B, C).
struct Fp64Launch {
  const double* A;
  const double* B;
  double* C;
  int64_t lda, ldb, ldc;
  int64_t a_rows, a_cols;  // extent of A that holds data (m x k); beyond reads as zero
  int64_t b_rows, b_cols;  // extent of B (k x n)
  int64_t c_rows, c_cols;  // extent of C that may be written (m x n, or hm x hn for M)
  int64_t hm, hn, hk;      // block edges
  int levels;
  int prod_begin, nprod;   // nprod < 0: all products of the level
  int m_target;            // 1: every product writes block (0,0) of C with sign + (temporary M)
  EpilogueKind epi;
  ScheduleKind sched;
  int tile;                // 0: 128 x 128 block tile, 1: 64 x 64, -1: the library's choice
  int trans_a, trans_b;    // op(A) = A^T (A stored k x m, ld >= m); op(B) = B^T (stored n x k)
  double alpha;            // C += alpha * (product); 1 for the plain operation
  int tri;                 // level 0 only: 0 every element of C, 1 only j <= i, 2 only j >= i
  int inner_targets;       // levels >= 2: scatter with the (levels-1)-level table's C coefficients
                           // (the inner products of the hybrid plan), blocks of hm x hn in C
};

// Fills the fields common to a full-operand launch.
Fp64Launch make_launch(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, int levels);

// Launches the FP64 product kernel on one problem; returns a CUDA error code.
cudaError_t launch_fp64(const Fp64Launch& L, cudaStream_t stream);

// Launches one persistent kernel over `count` problems (all scheduled stream-K with
// atomic C updates).  `scratch` is device memory of fp64_batched_scratch_bytes(count).
size_t fp64_batched_scratch_bytes(int count);
cudaError_t launch_fp64_batched(const Fp64Launch* probs, int count, void* scratch, cudaStream_t stream);

// Estimated busiest-SM time (FMA-equivalents) of one problem under a tile id and the
// stream-K schedule on `sms` blocks: the quantity the tile choices minimise.
double fp64_launch_estimate(const Fp64Launch& L, int tile_id, int sms);

// Launches one thread that waits on an mbarrier nothing completes, for `limit_cycles`
// clock cycles: exercises the bounded-wait path (the status word becomes
// STRASSEN_ERR_TIMEOUT and the kernel returns).
cudaError_t launch_wait_timeout_check(long long limit_cycles, cudaStream_t stream);

// Counts, over `count` hashed pairs, where the integer-pipe addition (int_fadd.h)
// differs bitwise from the hardware DADD on this device; synchronises `stream`.
cudaError_t check_int_fadd(long long count, unsigned long long seed, unsigned long long* mismatches_host,
                           cudaStream_t stream);

// Picks the tile (when L->tile < 0) and the schedule of a launch (balance heuristics
// for the SM count).
void choose_fp64_schedule(Fp64Launch* L, int prefer_deterministic);

// Length along k of one partial sum of the FP64 product kernel (a multiple of its
// k-step of 8): each consumer thread adds at most this many products in sequence
// before the partial sum leaves its registers for C (or M).  Shorter chunks cut the
// rounding error of long sums (which grows with the sequence length) at the cost of
// more C updates per tile; deeper tables get shorter chunks, their products being
// sums of more terms.
inline int accumulation_chunk_k(int levels) { return levels >= 3 ? 128 : 256; }

// Tile edge of a tile id (0: 128, 1: 64) and the number of tile ids.
constexpr int kNumTiles = 2;
inline int tile_edge_of(int tile_id) { return tile_id == 0 ? 128 : 64; }
// Cost of a 64 x 64 tile's multiply-adds relative to a 128 x 128 tile's, used by the
// tile choice and the model.  Its producers stage twice as many source elements per
// FMA: invisible up to two levels (measured 1.00-1.01), but the up-to-eight-term sums
// of three levels make the producers the bottleneck (measured 1.24).
inline double small_tile_factor(int levels) { return levels >= 3 ? 1.24 : 1.01; }

// Reads and clears the device-side status word of the product kernels (set when a
// bounded wait gave up).  Synchronises `stream` first.
int fp64_device_status(cudaStream_t stream);

// Naive / AB helpers (elementwise.cu).
// dst (rows x cols, ld = cols) = sum_t sign_t * block_t of src, masked to src's extent.
// With trans, src holds the transpose (element (r, c) at src[c * ld + r]).
cudaError_t launch_block_sum(double* dst, int64_t rows, int64_t cols,
                             const double* src, int64_t ld, int64_t src_rows, int64_t src_cols,
                             int64_t h_r, int64_t h_c, const uint8_t* terms, int nterms,
                             cudaStream_t stream, int trans = 0);
// For each target t: C block (bi, bj) += sign * alpha * M (hm x hn, ld = hn), masked to C.
cudaError_t launch_combine(double* C, int64_t ldc, int64_t c_rows, int64_t c_cols,
                           const double* M, int64_t hm, int64_t hn,
                           const uint8_t* targets, int ntargets, cudaStream_t stream, double alpha = 1.0);
// C (rows x cols, ldc) = beta C; beta = 0 writes zeros without reading C; beta = 1 is a no-op.
// With tri = 1 (2) only the elements with j <= i (j >= i) are scaled.
cudaError_t launch_scale(double* C, int64_t ldc, int64_t rows, int64_t cols, double beta, cudaStream_t stream,
                         int tri = 0);

int device_sm_count();

// Split-precision products (ozaki.cu): workspace bytes, the launch sequence (split,
// tensor-core slice products, recombine + scatter) on caller-provided workspace, and
// the read-and-clear of its device status word.
int64_t ozaki_workspace_bytes(int64_t m, int64_t n, int64_t k, int levels);
// With stage_events (four events), records them before the splits, before and after
// the slice products, and after the recombination.
cudaError_t run_ozaki(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
                      double* C, int64_t ldc, int levels, void* ws, cudaStream_t stream, int trans_a = 0,
                      int trans_b = 0, double alpha = 1.0, cudaEvent_t* stage_events = nullptr);
int ozaki_device_status();
// Analytic time of a split-precision call (the selector's model for that dtype).
double ozaki_model_seconds(int64_t m, int64_t n, int64_t k, int levels);

// Learned selector (mlp.cu).  Candidates: c = 0, 1 classical with tile c; c = 2 + 6 (L - 1)
// + 2 v + t: L levels (1, 2) of variant v (ABC, AB, Naive) with tile t; c = 14 + t: three
// levels of ABC with tile t.  The split-precision dtype takes the tile-0 ABC candidates
// only (0, 2, 8, 14: levels 0..3).
constexpr int kSelCandidates = 16;
constexpr int kSelInputs = 6 + kSelCandidates;
void selector_candidate(int c, int* levels, int* variant, int* tile);
bool selector_candidate_valid(int c, int dtype);
// Network inputs x[kSelInputs] and the analytic model's log2 seconds base[kSelCandidates].
void selector_features(int64_t m, int64_t n, int64_t k, int dtype, float* x, float* base);
// Argmin over the valid candidates of base + the loaded MLP's correction, for a shape;
// false when no network is loaded or enabled for the dtype, it lives on another device,
// or `may_launch` is 0 and the shape's choice is not cached (the first choice for a
// shape launches the select kernel and waits for it; later ones come from a host cache).
bool mlp_select(int64_t m, int64_t n, int64_t k, int dtype, int may_launch, int* candidate);

// Selection (select.cpp): analytic time model, its argmin, and the exhaustive records.
double model_seconds(int64_t m, int64_t n, int64_t k, int levels, int variant, int tile);
double model_seconds_dtype(int64_t m, int64_t n, int64_t k, int levels, int variant, int tile, int dtype);
void model_select(int64_t m, int64_t n, int64_t k, int* levels, int* variant, int* tile);
bool record_lookup(int64_t m, int64_t n, int64_t k, int dtype, int* levels, int* variant, int* tile);
void record_store(int64_t m, int64_t n, int64_t k, int dtype, int levels, int variant, int tile);
void record_clear();

}  // namespace sgb
