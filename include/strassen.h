/*
 * strassen.h -- C ABI of the GB300 (sm_103a) Strassen-fused GEMM library.
 *
 * The library implements the family of Strassen implementations of Huang, Smith,
 * Henry and van de Geijn, "Implementing Strassen's Algorithm with BLIS" (FLAME
 * Working Note #79, arXiv:1605.01078):
 *
 *   - the general operation of Eq. 1 / Eq. 3 / Eq. 4 (Sections 3.4-3.6): for every
 *     row r of the L-level coefficient table,
 *         M_r = (sum_s delta_s X_s)(sum_t eps_t V_t);   C_q += gamma_q M_r,
 *     with X_s blocks of A, V_t blocks of B, C_q blocks of C in a 2^L x 2^L partition;
 *   - the one-level table of Figure 1, the two-level table of Figure 2 (its
 *     Kronecker square) and the three-level table (its Kronecker cube: the
 *     multi-level Strassen of Sections 3.5-3.6 one level further);
 *   - the three variants of Section 4.1: "ABC" (operand sums formed while operand
 *     tiles are staged, each M_r scattered into its C blocks in the kernel
 *     epilogue), "AB" (fused sums, explicit temporary M, separate C updates) and
 *     "Naive" (explicit operand-sum temporaries, a classical GEMM, separate C
 *     updates).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Operation:  C <- C + A * B  (alpha = beta = 1; the paper reduces DGEMM to
 *             C = alpha*A*B + C in Section 2.2).  strassen_dgemm adds the full BLAS
 *             form C = alpha op(A) op(B) + beta C with transposes.
 * Layout:     row-major.  A is m x k with lda >= k, B is k x n with ldb >= n, C is
 *             m x n with ldc >= n; element (i, j) of A is A[i*lda + j].  Column-major
 *             callers pass (B^T, A^T, C^T) with m and n swapped.
 * Memory:     A, B, C are DEVICE pointers owned by the caller, 8-byte aligned; C must
 *             not overlap A or B.  Calls are asynchronous on `stream` (a
 *             cudaStream_t; NULL = the legacy default stream).  Unless stated
 *             otherwise the library allocates nothing for ABC and classical calls;
 *             AB and Naive take stream-ordered temporaries (cudaMallocAsync /
 *             cudaFreeAsync on `stream`) of strassen_workspace_size() bytes.
 * Sizes:      m, n, k >= 0; a call with m, n or k equal to 0 does nothing and
 *             returns STRASSEN_OK.  Odd and non-power-of-two sizes are handled by
 *             virtual zero padding: block i of a dimension d spans
 *             [i*h, min((i+1)*h, d)) with h = ceil(d / 2^L) (Section 3.3).
 * Errors:     every function returns STRASSEN_OK (0) or a negative status; nothing
 *             throws, exits or traps.  Invalid arguments are rejected on the host
 *             before anything is launched.  STRASSEN_ERR_CUDA reports a CUDA error
 *             seen by the call (launch failure or an earlier asynchronous error).
 * Numbers:    FP64 in and out.  For the split-precision dtypes the products run on
 *             the tensor cores on integer slices of the FP64 operands (see
 *             strassen_dtype) and the scaling, recombination and C accumulation stay
 *             in FP64.
 * Levels:     0 (classical) to STRASSEN_MAX_LEVELS = 3 (343 products); the FP64 kernel
 *             picks a 128x128 or 64x64 block tile per call (strassen_select reports
 *             the tile it would use: tile_id 0 or 1).
 */
#ifndef STRASSEN_GB300_H
#define STRASSEN_GB300_H

#include <stdint.h>
#include <stddef.h>

#if defined(__GNUC__)
#define STRASSEN_API __attribute__((visibility("default")))
#else
#define STRASSEN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef void* strassen_stream_t; /* a cudaStream_t */

/* Implementation variant (Section 4.1, "Variations on a theme"). */
typedef enum {
  STRASSEN_ABC = 0,   /* sums fused into operand staging, M_r scattered into C in the epilogue */
  STRASSEN_AB = 1,    /* sums fused into operand staging, M_r to a temporary, then C updates */
  STRASSEN_NAIVE = 2, /* operand-sum temporaries, classical GEMM into M_r, then C updates */
  STRASSEN_AUTO = 3,  /* chosen by strassen_select() */
  STRASSEN_HYBRID = 4 /* AB at the outermost level over ABC for the levels below it (levels >= 2;
                         at one level it is AB): see strassen_gemm */
} strassen_variant;

/* Arithmetic of the products. */
typedef enum {
  STRASSEN_F64 = 0,         /* FP64 fused multiply-adds */
  STRASSEN_F64_OZ_INT8 = 1, /* FP64 emulated by exact products of INT8 slices (INT32 accumulation) */
  STRASSEN_F64_OZ_BF16 = 2  /* FP64 emulated by exact products of BF16 integer slices (FP32 accumulation, k-chunked) */
} strassen_dtype;

/* Status codes. */
#define STRASSEN_OK 0
#define STRASSEN_ERR_DIM (-1)         /* m, n or k negative */
#define STRASSEN_ERR_LD (-2)          /* lda < k, ldb < n or ldc < n (with a non-empty operand) */
#define STRASSEN_ERR_NULL (-3)        /* NULL pointer with a non-empty operand */
#define STRASSEN_ERR_LEVELS (-4)      /* levels outside {-1, 0, 1, 2, 3} */
#define STRASSEN_MAX_LEVELS 3         /* deepest table built: 7^3 = 343 products */
#define STRASSEN_MAX_TERMS 8          /* terms per operand / C targets per product (2^3) */
#define STRASSEN_ERR_UNSUPPORTED (-5) /* unknown dtype or variant, or a combination not built */
#define STRASSEN_ERR_CUDA (-6)        /* a CUDA runtime error */
#define STRASSEN_ERR_TIMEOUT (-7)     /* a device-side wait gave up (batched work queue) */
#define STRASSEN_ERR_ALLOC (-8)       /* a temporary could not be allocated */
#define STRASSEN_ERR_ARG (-9)         /* any other invalid argument (count, pointer array, ...) */
#define STRASSEN_ERR_SCRATCH_LIMIT (-10) /* the product needs more than the fixed scratch array of
                                            strassen_gemm_ab_noalloc holds */

/*
 * strassen_gemm -- C += A*B with `levels` levels of Strassen in `variant`.
 *
 * Defined by Eq. 4 (Section 3.6) with the Figure 1 table (levels = 1), its
 * Kronecker square, Figure 2 (levels = 2), or its Kronecker cube (levels = 3, 343
 * products); levels = 0 is the classical product of Section 2.1.  levels = -1 or variant = STRASSEN_AUTO asks strassen_select() for the
 * choice.  Levels are clamped down while 2^levels exceeds min(m, n, k) (a block would
 * be empty in every product); the call still succeeds.
 *
 *   m, n, k       sizes (>= 0); A m x k, B k x n, C m x n, row-major.
 *   A, lda        device pointer and row stride (elements) of A, lda >= max(k, 1).
 *   B, ldb        device pointer and row stride of B, ldb >= max(n, 1).
 *   C, ldc        device pointer and row stride of C, ldc >= max(n, 1); read and written.
 *   levels        -1 (auto), 0, 1, 2 or 3.
 *   variant       STRASSEN_ABC, STRASSEN_AB, STRASSEN_NAIVE, STRASSEN_HYBRID or STRASSEN_AUTO.
 *   dtype         STRASSEN_F64 or one of the split-precision dtypes.
 *   stream        the CUDA stream the work is ordered on.
 *
 * Returns STRASSEN_OK or a negative status; on error C is untouched unless the status
 * is STRASSEN_ERR_CUDA (work may have been partly launched).  ABC in FP64 with the
 * default scheduling accumulates the partial products into C with device atomics, so
 * the rounding order (not the mathematical result) can vary from run to run;
 * strassen_dgemm_ex with STRASSEN_FLAG_DETERMINISTIC makes every C tile owned by one
 * thread block, which fixes the order (at some cost in load balance).
 *
 * Hybrid plans (Eq. 4 applied with different variants at different levels): with
 * STRASSEN_HYBRID and L >= 2 levels the outermost level is AB and the L-1 levels below
 * it are ABC: for each of the 7 outer products a, one launch runs its 7^(L-1) inner
 * products with fused operand sums (the L-level table's terms) and scatters them, in
 * the epilogue, into the quadrants of a temporary M_a of (2^(L-1) ceil(m/2^L)) x
 * (2^(L-1) ceil(n/2^L)) doubles with the inner table's coefficients; a separate pass
 * then adds gamma M_a into the C blocks of outer product a.  (The other mix, ABC over
 * AB, is the L-level AB variant itself: its temporaries are scattered with the
 * composite coefficients.)  The temporary is stream-ordered, as for AB.
 *
 * Accuracy: each FP64 partial product is accumulated over at most 256 of k (128 at
 * three levels) in registers and then added into C (or M), so no sequential sum is
 * longer than that chunk plus the number of chunks and products per C element.
 */
STRASSEN_API int strassen_gemm(int64_t m, int64_t n, int64_t k,
                  const double* A, int64_t lda,
                  const double* B, int64_t ldb,
                  double* C, int64_t ldc,
                  int levels, strassen_variant variant, strassen_dtype dtype,
                  strassen_stream_t stream);

/*
 * classical_gemm -- C += A*B by the classical definition of Section 2.1
 * (gamma_ij += sum_p alpha_ip beta_pj), in FP64 on the library's own kernel.
 * Arguments, layout, ownership and errors as strassen_gemm.  Each C tile is owned by
 * one thread block unless splitting k is needed to fill the GPU, in which case the
 * partial sums are accumulated with device atomics.
 */
STRASSEN_API int classical_gemm(int64_t m, int64_t n, int64_t k,
                   const double* A, int64_t lda,
                   const double* B, int64_t ldb,
                   double* C, int64_t ldc,
                   strassen_stream_t stream);

/*
 * strassen_dgemm -- the full BLAS operation C = alpha op(A) op(B) + beta C with the
 * Strassen family, so the library can stand in for a DGEMM call (the paper's reduction
 * of DGEMM to C = alpha A B + C in Section 2.2 and its plug-compatibility aim of
 * Section 1; row-major here, as everywhere in this library).
 *
 *   transa, transb   0: op(X) = X; 1: op(X) = X^T.  op(A) is m x k, op(B) is k x n.
 *   A, lda           stored m x k (lda >= k) when transa = 0, k x m (lda >= m) when 1.
 *   B, ldb           stored k x n (ldb >= n) when transb = 0, n x k (ldb >= k) when 1.
 *   alpha, beta      scalars.  beta = 0 sets C to alpha op(A) op(B) without reading C
 *                    (NaNs in C do not propagate); alpha = 0 or k = 0 only scales C.
 *   C, ldc           m x n, ldc >= n; must not overlap A or B.
 *   levels, variant, dtype, stream   as strassen_gemm (levels -1 / STRASSEN_AUTO choose).
 *
 * Order of operations: C = beta C (one multiply per element, skipped for beta = 1),
 * then the product is added as in strassen_gemm with every partial product M_r scaled
 * by alpha where it is added into C (the epilogue of ABC, the C updates of AB and
 * Naive, the recombination of the split-precision path): for alpha = beta = 1 and no
 * transposes the result is that of strassen_gemm.  Transposed operands are read in
 * place (no copies): the FP64 kernel loads their tiles with the other box orientation.
 * Returns STRASSEN_OK or a negative status (STRASSEN_ERR_ARG for transa or transb
 * outside {0, 1}).
 */
STRASSEN_API int strassen_dgemm(int transa, int transb, int64_t m, int64_t n, int64_t k, double alpha,
                                const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                                double* C, int64_t ldc, int levels, strassen_variant variant,
                                strassen_dtype dtype, strassen_stream_t stream);

/* Flags of strassen_dgemm_ex. */
#define STRASSEN_FLAG_DETERMINISTIC 1u /* fixed rounding order: bitwise the same result on every run */

/*
 * strassen_dgemm_ex -- strassen_dgemm with options.  Arguments as strassen_dgemm, plus
 *
 *   flags   0 or STRASSEN_FLAG_DETERMINISTIC.  With the flag, every FP64 product
 *           launch (ABC, the product kernels of AB and Naive, classical) gives each C
 *           tile (or tile of the temporary M) to one thread block, which adds the
 *           partial products of every element in one fixed order (products in table
 *           order, k chunks in ascending order): the same inputs give bitwise the same
 *           C on every run and every GPU of the same kind.  Without it the library may
 *           split the k range of a tile over blocks (stream-K) for load balance, and
 *           the order of the atomic C additions then varies.  The split-precision path
 *           is deterministic either way.  Other bits: STRASSEN_ERR_ARG.
 *
 * strassen_gemm(...) is strassen_dgemm_ex(0, 0, ..., alpha 1, beta 1, ..., flags 0).
 */
STRASSEN_API int strassen_dgemm_ex(int transa, int transb, int64_t m, int64_t n, int64_t k, double alpha,
                                   const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                                   double* C, int64_t ldc, int levels, strassen_variant variant,
                                   strassen_dtype dtype, unsigned flags, strassen_stream_t stream);

/*
 * strassen_dsyrk -- the symmetric rank-k update C = alpha op(A) op(A)^T + beta C on one
 * triangle of C (the BLAS DSYRK operation, row-major), with the Strassen family doing
 * the off-diagonal products: the paper's conclusion names the other level-3 BLAS
 * operations as users of the same fused Strassen kernels.
 *
 *   uplo     0: the lower triangle (j <= i, diagonal included) is updated; 1: the upper
 *            (j >= i).  Elements of C outside that triangle are neither read nor written.
 *   trans    0: op(A) = A, A stored n x k (lda >= k); 1: op(A) = A^T, A stored k x n
 *            (lda >= n).  Transposed operands are read in place.
 *   n, k     C is n x n (ldc >= n); k >= 0.
 *   alpha, beta   beta = 0 sets the triangle to alpha op(A) op(A)^T without reading it;
 *            alpha = 0 or k = 0 only scales the triangle.
 *   levels   Strassen levels of the off-diagonal products (-1: the selector's choice for
 *            each product); the diagonal blocks are classical.
 *   flags    0 or STRASSEN_FLAG_DETERMINISTIC (as strassen_dgemm_ex).
 *
 * Method: the triangle is scaled by beta; then, recursively, C = [C00 .; C10 C11] (lower)
 * with a split n0 near n/2 (a multiple of 128 where possible): C00 and C11 by the same
 * recursion, C10 += alpha op(A)[n0:] op(A)[:n0]^T by the Strassen product (the upper
 * triangle takes C01 instead); blocks of at most 1024 rows are one classical launch whose
 * epilogue writes only the triangle.  C must not overlap A.  Returns STRASSEN_OK or a
 * negative status (STRASSEN_ERR_ARG for uplo, trans or flags outside their values).
 */
STRASSEN_API int strassen_dsyrk(int uplo, int trans, int64_t n, int64_t k, double alpha, const double* A,
                                int64_t lda, double beta, double* C, int64_t ldc, int levels, unsigned flags,
                                strassen_stream_t stream);

/* One problem of a batched call: C += A*B as in strassen_gemm. */
typedef struct {
  int64_t m, n, k;
  const double* A;
  const double* B;
  double* C;
  int64_t lda, ldb, ldc;
  int levels;               /* -1 = the autotuner's choice, else 0, 1, 2 or 3 */
  strassen_variant variant; /* STRASSEN_ABC or STRASSEN_AUTO (both run the fused ABC form);
                               AB and Naive only with levels = 0 (classical) */
} strassen_problem;

/*
 * strassen_gemm_batched -- many independent products of uneven shapes in persistent
 * kernel launches (the batching pattern; not in the paper).
 *
 *   count   number of problems (>= 0).
 *   probs   HOST array of `count` problems; each is validated as in strassen_gemm.
 *           The byte ranges [C, C + (m-1)*ldc + n) of different problems must not
 *           overlap (STRASSEN_ERR_ARG otherwise).  Every problem runs as ABC
 *           (levels 1-3) or classical (levels 0); a problem asking for AB or Naive
 *           with levels other than 0 returns STRASSEN_ERR_UNSUPPORTED.  Each problem
 *           gets the block tile (128x128 or 64x64) with the smaller estimate of padded
 *           tile work, and with levels = -1 also the level (an exhaustive record for
 *           the shape, strassen_tune_record, takes precedence).
 *   dtype   STRASSEN_F64.
 *   stream  the CUDA stream.
 *
 * Problems with the same tile share one persistent launch, so the call makes one launch
 * per tile in use (at most two).  Within a launch the thread blocks claim whole work
 * units (problem, product, output tile, all of its k) from a counter, problems with the
 * longest units first, and add their partial products into C with device atomics.
 * With two launches the larger goes first on `stream` and the other on a library stream
 * forked from it with an event (so one launch's tail overlaps the other's start);
 * `stream` waits for both before the call's work counts as done.  The work list travels in kernel parameters
 * to a small kernel that writes it into a stream-ordered temporary (cudaMallocAsync),
 * so the whole call can be captured in a CUDA graph and replayed; make one call on the
 * device outside a capture first (it creates the library stream).  Returns STRASSEN_OK
 * or a negative status.
 */
STRASSEN_API int strassen_gemm_batched(int count, const strassen_problem* probs,
                          strassen_dtype dtype, strassen_stream_t stream);

/*
 * strassen_select -- the variant selector: picks which member of the family (classical,
 * or 1 / 2 / 3 levels of ABC, AB or Naive) and which block tile (tile_id 0: 128x128x8,
 * 1: 64x64x8) to run for an m x n x k product in `dtype` -- the choice Section 4.2 of
 * the paper builds its performance model for.  In order of precedence it returns
 *   1. the exhaustive-measurement record for exactly this shape and dtype, if one was
 *      stored with strassen_tune_record();
 *   2. the argmin of the learned selector's predictions over its 16 candidates (levels
 *      0-2 of every variant and three-level ABC, each with both tiles; see
 *      strassen_selector_candidate), if a network was
 *      loaded with strassen_selector_load() and is enabled for the dtype.  The first
 *      choice for a shape runs one small kernel on a library stream and waits for it;
 *      the choice is cached, so later calls for the shape do no GPU work;
 *   3. the analytic model's argmin over levels 0 to 3, variants and tiles otherwise
 *      (FP64), or classical slices (split-precision dtypes).
 * strassen_gemm with levels = -1 and STRASSEN_AUTO runs exactly the selected
 * (levels, variant, tile); inside a stream capture it uses the learned selector only for
 * shapes already in its cache (no launch, no wait) and otherwise the model.
 * The model prefers fewer levels on ties within 1 %.
 *
 *   levels, variant, tile_id   outputs (host pointers, non-NULL).
 * Returns STRASSEN_OK or a negative status.
 */
STRASSEN_API int strassen_select(int64_t m, int64_t n, int64_t k, strassen_dtype dtype,
                                 int* levels, strassen_variant* variant, int* tile_id);

/*
 * strassen_tune_record / strassen_tune_clear -- store (or forget all) exhaustive
 * measurement results: the fastest (levels 0-3, variant, tile_id 0 or 1) measured for
 * a shape and dtype, which strassen_select() then returns for exactly that shape.  The
 * table lives in host memory of the process.  Returns STRASSEN_OK or a negative status.
 */
STRASSEN_API int strassen_tune_record(int64_t m, int64_t n, int64_t k, strassen_dtype dtype,
                                      int levels, strassen_variant variant, int tile_id);
STRASSEN_API int strassen_tune_clear(void);

/*
 * strassen_model_seconds -- the analytic time model (the paper's T = T_a + T_m of
 * Section 4.2, restated for this GPU): FP64 multiply-adds of the padded block tiles
 * (the cheaper of 128x128x8 and 64x64x8) and the additions of Naive's and AB's separate
 * kernels at the FP64 pipe rate (ABC's and AB's staging sums run on the integer pipe),
 * the extra temporary passes of AB and Naive at the HBM rate, and a fixed cost per
 * kernel launch.  Returns the predicted seconds, or -1 for invalid arguments.
 */
STRASSEN_API double strassen_model_seconds(int64_t m, int64_t n, int64_t k, int levels,
                                           strassen_variant variant);

/*
 * The learned selector (not in the paper; it stands in for the analytic model of
 * Section 4.2).  A multilayer perceptron 22 -> 64 -> 64 -> 16 (FP32, ReLU) maps a
 * shape's features to a correction of the analytic model's log2 seconds for each of
 * STRASSEN_SELECTOR_CANDIDATES = 16 candidates; the selection is the argmin over the
 * dtype's valid candidates of (model log2 seconds + correction).  Features, from
 * strassen_selector_features: (log2 m - 11)/3, (log2 n - 11)/3, (log2 k - 11)/3, dtype
 * one-hot, then for every candidate (model log2 seconds + 7)/7.  Candidates
 * (strassen_selector_candidate): 0, 1 classical with tile 0, 1; 2 + 6 (L - 1) + 2 v + t
 * for L levels (1, 2), variant v (ABC, AB, Naive) and tile t; 14 + t three-level ABC.
 * The split-precision dtype uses the tile-0 ABC candidates (0, 2, 8, 14: levels 0-3).
 * Its parameters are one float vector of strassen_mlp_param_count() entries:
 * [W1 (64x22 row-major), b1 (64), W2 (64x64), b2 (64), W3 (16x64), b3 (16)].
 *
 * strassen_mlp_forward   Y[batch][16] = network(X[batch][22]); all DEVICE pointers.
 * strassen_mlp_loss_grad grad = d/dparams of sum mask (Y - T)^2 / mask_sum over the
 *                        batch (X [batch][22], T and mask [batch][16], DEVICE); grad is
 *                        overwritten.  mask_sum > 0 is the sum of mask.  For training,
 *                        T = log2 measured seconds - the model's log2 seconds.
 * strassen_mlp_adam      one Adam step (beta1 0.9, beta2 0.999, eps 1e-8; step >= 1)
 *                        on `count` parameters with moment buffers m, v (DEVICE).
 * strassen_selector_load keeps a copy of a trained parameter vector (HOST) and makes
 *                        strassen_select() use it on every device: the current device
 *                        gets its device copy at once, any other device on its first
 *                        selection (outside a stream capture); strassen_selector_clear
 *                        forgets it (and re-enables every dtype).
 * strassen_selector_use  enables (1) or disables (0) the network for one dtype
 *                        (default: all enabled); with it disabled, strassen_select()
 *                        falls through to the analytic model for that dtype.  The tuning
 *                        driver enables it only where it beat the model on held-out shapes.
 * strassen_selector_candidate  (levels, variant, tile_id) of candidate c (0..15).
 * strassen_selector_features   x[22] (network inputs), base[16] (the model's log2
 *                        seconds) and the bit mask of the candidates valid for `dtype`,
 *                        on the host (no GPU work; the model reads the device's SM
 *                        count and clock).
 * All return STRASSEN_OK or a negative status; the kernels run on `stream`.
 */
#define STRASSEN_SELECTOR_CANDIDATES 16
#define STRASSEN_SELECTOR_INPUTS 22
STRASSEN_API int strassen_mlp_param_count(void);
STRASSEN_API int strassen_mlp_forward(const float* params, const float* X, int batch, float* Y,
                                      strassen_stream_t stream);
STRASSEN_API int strassen_mlp_loss_grad(const float* params, const float* X, const float* T,
                                        const float* mask, int batch, float mask_sum, float* grad,
                                        strassen_stream_t stream);
STRASSEN_API int strassen_mlp_adam(float* params, const float* grad, float* m, float* v, int count,
                                   int step, float lr, strassen_stream_t stream);
STRASSEN_API int strassen_selector_load(const float* params_host, int count);
STRASSEN_API int strassen_selector_use(int dtype, int enable);
STRASSEN_API int strassen_selector_clear(void);
STRASSEN_API int strassen_selector_candidate(int candidate, int* levels, strassen_variant* variant,
                                             int* tile_id);
STRASSEN_API int strassen_selector_features(int64_t m, int64_t n, int64_t k, strassen_dtype dtype, float* x,
                                            float* base, unsigned* valid);

/*
 * strassen_workspace_size -- bytes of stream-ordered temporaries a strassen_gemm call
 * with these arguments takes (0 for ABC and classical in FP64).  AB needs one
 * (m/2^L) x (n/2^L) temporary M (Section 5, conclusion); Naive adds the operand sums.
 * Returns a negative status for invalid arguments.
 */
STRASSEN_API int64_t strassen_workspace_size(int64_t m, int64_t n, int64_t k, int levels,
                                strassen_variant variant, strassen_dtype dtype);

/*
 * strassen_gemm_ab_noalloc -- the AB variant (levels 1 to 3) that allocates nothing.
 * The paper has no counterpart: it is an interface for callers that cannot allocate
 * device memory while they run -- a process whose device memory is already claimed by
 * its own pooling allocator, a latency-bound loop where an allocation or a free may
 * synchronise the device, or code that must have no out-of-memory failure path.
 *
 * Computes C += A*B exactly as strassen_gemm(..., levels, STRASSEN_AB, STRASSEN_F64,
 * stream) does (same arguments, layout, ownership and checks), but the temporary
 * M_r of (ceil(m/2^L) x ceil(n/2^L)) doubles lives in one fixed array of 4 Mi doubles
 * (32 MiB) compiled into the library, so the call makes no cudaMalloc, cudaFree or
 * other allocating call.  Every GPU that loads the library holds that array until the
 * process exits.
 *
 *   Limit:   ceil(m/2^L) * ceil(n/2^L) <= 4194304 (e.g. m = n = 4096 at one level,
 *            8192 at two); larger products return STRASSEN_ERR_SCRATCH_LIMIT and touch
 *            nothing.  levels outside {1, 2, 3} return STRASSEN_ERR_LEVELS (levels are
 *            clamped as in strassen_gemm; a clamp to 0 runs classical_gemm).
 *   Set-up:  the first call on each device looks up the array's device address with
 *            cudaGetSymbolAddress while that device is current; make that first call
 *            before any stream capture.
 *   Sharing: all calls in the process share the one array and it keeps the last
 *            call's contents (the kernels overwrite or clear what they read).  Calls
 *            whose work overlaps on the GPU (different streams, or different host
 *            threads without ordering) race on the array and give wrong results:
 *            order them on one stream or synchronise between them.
 */
STRASSEN_API int strassen_gemm_ab_noalloc(int64_t m, int64_t n, int64_t k,
                                          const double* A, int64_t lda,
                                          const double* B, int64_t ldb,
                                          double* C, int64_t ldc,
                                          int levels, strassen_stream_t stream);

/*
 * strassen_device_status -- waits for `stream`, then reads and clears the library's
 * device status word.  The kernels bound every device-side wait (about one second);
 * a wait that runs out sets the word to STRASSEN_ERR_TIMEOUT and the kernel returns
 * instead of hanging.  Returns STRASSEN_OK, STRASSEN_ERR_TIMEOUT or STRASSEN_ERR_CUDA.
 */
STRASSEN_API int strassen_device_status(strassen_stream_t stream);

/*
 * strassen_check_wait_timeout -- diagnostic: launches one thread that waits on a
 * barrier nothing completes, for `limit_cycles` SM clock cycles, through the same
 * bounded-wait code the kernels use.  Afterwards strassen_device_status() returns
 * STRASSEN_ERR_TIMEOUT and the context stays usable.  Returns STRASSEN_OK or a
 * negative status (STRASSEN_ERR_ARG for a negative limit).
 */
STRASSEN_API int strassen_check_wait_timeout(int64_t limit_cycles, strassen_stream_t stream);

/*
 * strassen_check_int_fadd -- diagnostic: on the current device, adds and subtracts
 * `count` hashed pairs of doubles (arbitrary bit patterns, near-cancelling pairs,
 * subnormals, wide exponent gaps) both with the hardware FP64 addition and with the
 * integer-pipe addition the staging kernels use for operand sums, and stores in
 * *mismatches (HOST pointer) how many results differ bitwise.  Synchronises `stream`.
 * Returns STRASSEN_OK or a negative status.
 */
STRASSEN_API int strassen_check_int_fadd(int64_t count, uint64_t seed, uint64_t* mismatches,
                                         strassen_stream_t stream);

/*
 * strassen_profile_split_precision -- diagnostic: one split-precision product
 * C += A*B (strassen_gemm with dtype STRASSEN_F64_OZ_BF16, variant ABC, `levels` 0-3;
 * same arguments, layout and checks) with CUDA events between its three stages, then a
 * wait for the call.  stage_ms (HOST, 3 floats) receives the milliseconds of
 * [0] the operand splits (operand sums, scaling, digit extraction: three kernels),
 * [1] the tensor-core slice products (one kernel), [2] the recombination with the C
 * scatter (one kernel).  Returns STRASSEN_OK or a negative status.
 */
STRASSEN_API int strassen_profile_split_precision(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                                                  const double* B, int64_t ldb, double* C, int64_t ldc,
                                                  int levels, float* stage_ms, strassen_stream_t stream);

/* strassen_status_string -- a static, NUL-terminated description of a status code. */
STRASSEN_API const char* strassen_status_string(int status);

/*
 * strassen_plan_table -- copies the coefficient table the library uses for `levels`
 * (0 to STRASSEN_MAX_LEVELS) into host arrays, for inspection and tests; no GPU work.
 *
 * Each of the 7^levels products r has up to 2^levels terms per operand.  Term t of
 * product r is stored at index r*STRASSEN_MAX_TERMS + t of a_terms, b_terms, c_terms
 * as (block_row * 16 + block_col) * 2 + (sign < 0) (unused entries -1), and the term
 * counts at na[r], nb[r], nc[r].  `capacity` is the number of products the arrays can
 * hold (a_terms etc. hold STRASSEN_MAX_TERMS*capacity ints).  Returns the number of
 * products, or a negative status.
 */
STRASSEN_API int strassen_plan_table(int levels, int capacity, int* na, int* nb, int* nc,
                        int* a_terms, int* b_terms, int* c_terms);

#ifdef __cplusplus
}
#endif

#endif /* STRASSEN_GB300_H */
