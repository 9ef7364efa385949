/*
 * CPU oracle for the GEMM / Strassen hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes, links or calls
 * this file; only the tests, the smoke check and the CPU leg of the benchmark (its
 * baseline timing and the reference entries of its error figures) load it.  It shares
 * no code, header or table with the CUDA path.
 *
 * Everything is plain IEEE double arithmetic, row-major, one thread, written to be
 * checked against the paper by eye rather than to be fast (a second build with OpenMP,
 * used only to time the oracle on all host cores, splits the rows of each classical
 * product over threads without changing any entry's arithmetic):
 *
 *   oracle_gemm          - the definition of C = alpha*A*B + C with alpha = 1
 *                          (Section 2.1): gamma_ij += sum_p alpha_ip * beta_pj.
 *   oracle_strassen      - textbook Strassen: the seven products of Figure 1
 *                          (Section 3.1), applied recursively (Section 3.2), with
 *                          explicit temporaries and zero padding of odd sizes
 *                          (Section 3.3), and the classical definition at the leaves.
 *   oracle_strassen_sampled - selected entries of oracle_strassen's result, computed
 *                          one by one in exactly its order of operations (for
 *                          products too large for the full recursion on a CPU).
 *   oracle_gemm_sampled  - selected entries of C0 + A*B computed with the compensated
 *                          dot product Dot2 of Ogita, Rump and Oishi, "Accurate sum and
 *                          dot product", SIAM J. Sci. Comput. 26(6), 2005 (Algorithm
 *                          5.3 there): the result is as accurate as if computed in
 *                          twice the working precision and then rounded.
 *
 * Parity pins (tests/test_oracle_*.py): integer-valued inputs give results that are
 * exact in double, so oracle_gemm and oracle_strassen must agree bit for bit with an
 * independent brute-force product; the multiply counter must give 7^L (h_m h_n h_k)
 * against 8^L; identity and permutation matrices give known results exactly; the
 * sampled Dot2 entries must equal exact rational products.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- classical */

/* C[i][j] += sum_{p=0}^{k-1} A[i][p] * B[p][j]; the sum over p is formed first, in
 * ascending p, then added to C[i][j] (the order the definition is written in).
 * B is copied once into a transposed buffer so that each dot product reads two
 * contiguous rows; this changes storage only, not the arithmetic.
 * Returns the number of scalar multiplications (m*n*k), or -1 if out of memory. */
int64_t oracle_gemm(int64_t m, int64_t n, int64_t k,
                    const double* A, int64_t lda,
                    const double* B, int64_t ldb,
                    double* C, int64_t ldc) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  double* Bt = (double*)malloc(sizeof(double) * (size_t)n * (size_t)k);
  if (!Bt) return -1;
  for (int64_t p = 0; p < k; ++p)
    for (int64_t j = 0; j < n; ++j) Bt[j * k + p] = B[p * ldb + j];
  /* Rows of C are independent; the timing build (OpenMP) splits them over threads,
   * the correctness build ignores this line.  Each entry's arithmetic is the same. */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    const double* a = A + i * lda;
    for (int64_t j = 0; j < n; ++j) {
      const double* b = Bt + j * k;
      double s = 0.0;
      for (int64_t p = 0; p < k; ++p) s += a[p] * b[p];
      C[i * ldc + j] += s;
    }
  }
  free(Bt);
  return m * n * k;
}

/* ---------------------------------------------------------------- Strassen */

/* A dense h_r x h_c block with its own storage (leading dimension h_c). */
typedef struct { int64_t r, c; double* v; } blk;

static blk blk_new(int64_t r, int64_t c) {
  blk b; b.r = r; b.c = c;
  b.v = (double*)calloc((size_t)(r * c > 0 ? r * c : 1), sizeof(double));
  return b;
}

/* Quadrant (qi, qj) of an R x Cc matrix X (leading dimension ldx) split with
 * h_r = ceil(R/2), h_c = ceil(Cc/2): rows [qi*h_r, min((qi+1)*h_r, R)), columns
 * likewise; entries past the edge of X are the zero padding of Section 3.3. */
static void quad_load(blk* dst, const double* X, int64_t ldx, int64_t R, int64_t Cc,
                      int qi, int qj) {
  for (int64_t i = 0; i < dst->r; ++i) {
    int64_t gi = qi * dst->r + i;
    for (int64_t j = 0; j < dst->c; ++j) {
      int64_t gj = qj * dst->c + j;
      dst->v[i * dst->c + j] = (gi < R && gj < Cc) ? X[gi * ldx + gj] : 0.0;
    }
  }
}

/* C quadrant (qi, qj) += sign * M, skipping the padded rows and columns. */
static void quad_update(double* C, int64_t ldc, int64_t R, int64_t Cc, int qi, int qj,
                        double sign, const blk* M) {
  for (int64_t i = 0; i < M->r; ++i) {
    int64_t gi = qi * M->r + i;
    if (gi >= R) break;
    for (int64_t j = 0; j < M->c; ++j) {
      int64_t gj = qj * M->c + j;
      if (gj >= Cc) break;
      C[gi * ldc + gj] += sign * M->v[i * M->c + j];
    }
  }
}

/* out = x + s*y (s = +1 or -1), elementwise. */
static void blk_add(blk* out, const blk* x, double s, const blk* y) {
  for (int64_t t = 0; t < out->r * out->c; ++t) out->v[t] = x->v[t] + s * y->v[t];
}

static void blk_copy(blk* out, const blk* x) {
  memcpy(out->v, x->v, sizeof(double) * (size_t)(out->r * out->c));
}

int64_t oracle_strassen(int levels, int64_t m, int64_t n, int64_t k,
                        const double* A, int64_t lda,
                        const double* B, int64_t ldb,
                        double* C, int64_t ldc);

/* M = S*T with (levels) more levels of Strassen; M starts at zero. */
static int64_t blk_mul(int levels, blk* M, const blk* S, const blk* T) {
  return oracle_strassen(levels, M->r, M->c, S->c, S->v, S->c, T->v, T->c, M->v, M->c);
}

/* C += A*B by one level of Figure 1 on top of (levels-1) further levels.  The seven
 * products and their C updates are written out in the figure's order and notation:
 *
 *   M0 = (A00 + A11)(B00 + B11);  C00 += M0;  C11 += M0;
 *   M1 = (A10 + A11) B00;         C10 += M1;  C11 -= M1;
 *   M2 = A00 (B01 - B11);         C01 += M2;  C11 += M2;
 *   M3 = A11 (B10 - B00);         C00 += M3;  C10 += M3;
 *   M4 = (A00 + A01) B11;         C01 += M4;  C00 -= M4;
 *   M5 = (A10 - A00)(B00 + B01);  C11 += M5;
 *   M6 = (A01 - A11)(B10 + B11);  C00 += M6;
 *
 * Returns the number of scalar multiplications, or -1 if out of memory. */
int64_t oracle_strassen(int levels, int64_t m, int64_t n, int64_t k,
                        const double* A, int64_t lda,
                        const double* B, int64_t ldb,
                        double* C, int64_t ldc) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  if (levels <= 0) return oracle_gemm(m, n, k, A, lda, B, ldb, C, ldc);
  const int64_t hm = (m + 1) / 2, hn = (n + 1) / 2, hk = (k + 1) / 2;
  blk A00 = blk_new(hm, hk), A01 = blk_new(hm, hk), A10 = blk_new(hm, hk), A11 = blk_new(hm, hk);
  blk B00 = blk_new(hk, hn), B01 = blk_new(hk, hn), B10 = blk_new(hk, hn), B11 = blk_new(hk, hn);
  blk S = blk_new(hm, hk), T = blk_new(hk, hn), M = blk_new(hm, hn);
  int64_t mults = 0, r;
  int oom = !A00.v || !A01.v || !A10.v || !A11.v || !B00.v || !B01.v || !B10.v ||
            !B11.v || !S.v || !T.v || !M.v;
  if (!oom) {
    quad_load(&A00, A, lda, m, k, 0, 0); quad_load(&A01, A, lda, m, k, 0, 1);
    quad_load(&A10, A, lda, m, k, 1, 0); quad_load(&A11, A, lda, m, k, 1, 1);
    quad_load(&B00, B, ldb, k, n, 0, 0); quad_load(&B01, B, ldb, k, n, 0, 1);
    quad_load(&B10, B, ldb, k, n, 1, 0); quad_load(&B11, B, ldb, k, n, 1, 1);
  }
#define PRODUCT(stmt_s, stmt_t)                                        \
  do {                                                                 \
    stmt_s; stmt_t;                                                    \
    memset(M.v, 0, sizeof(double) * (size_t)(hm * hn));                \
    r = blk_mul(levels - 1, &M, &S, &T);                               \
    if (r < 0) { oom = 1; break; }                                     \
    mults += r;                                                        \
  } while (0)
  if (!oom) {
    /* M0 = (A00 + A11)(B00 + B11); C00 += M0; C11 += M0 */
    PRODUCT(blk_add(&S, &A00, +1, &A11), blk_add(&T, &B00, +1, &B11));
    if (!oom) { quad_update(C, ldc, m, n, 0, 0, +1, &M); quad_update(C, ldc, m, n, 1, 1, +1, &M); }
  }
  if (!oom) {
    /* M1 = (A10 + A11) B00; C10 += M1; C11 -= M1 */
    PRODUCT(blk_add(&S, &A10, +1, &A11), blk_copy(&T, &B00));
    if (!oom) { quad_update(C, ldc, m, n, 1, 0, +1, &M); quad_update(C, ldc, m, n, 1, 1, -1, &M); }
  }
  if (!oom) {
    /* M2 = A00 (B01 - B11); C01 += M2; C11 += M2 */
    PRODUCT(blk_copy(&S, &A00), blk_add(&T, &B01, -1, &B11));
    if (!oom) { quad_update(C, ldc, m, n, 0, 1, +1, &M); quad_update(C, ldc, m, n, 1, 1, +1, &M); }
  }
  if (!oom) {
    /* M3 = A11 (B10 - B00); C00 += M3; C10 += M3 */
    PRODUCT(blk_copy(&S, &A11), blk_add(&T, &B10, -1, &B00));
    if (!oom) { quad_update(C, ldc, m, n, 0, 0, +1, &M); quad_update(C, ldc, m, n, 1, 0, +1, &M); }
  }
  if (!oom) {
    /* M4 = (A00 + A01) B11; C01 += M4; C00 -= M4 */
    PRODUCT(blk_add(&S, &A00, +1, &A01), blk_copy(&T, &B11));
    if (!oom) { quad_update(C, ldc, m, n, 0, 1, +1, &M); quad_update(C, ldc, m, n, 0, 0, -1, &M); }
  }
  if (!oom) {
    /* M5 = (A10 - A00)(B00 + B01); C11 += M5 */
    PRODUCT(blk_add(&S, &A10, -1, &A00), blk_add(&T, &B00, +1, &B01));
    if (!oom) quad_update(C, ldc, m, n, 1, 1, +1, &M);
  }
  if (!oom) {
    /* M6 = (A01 - A11)(B10 + B11); C00 += M6 */
    PRODUCT(blk_add(&S, &A01, -1, &A11), blk_add(&T, &B10, +1, &B11));
    if (!oom) quad_update(C, ldc, m, n, 0, 0, +1, &M);
  }
#undef PRODUCT
  free(A00.v); free(A01.v); free(A10.v); free(A11.v);
  free(B00.v); free(B01.v); free(B10.v); free(B11.v);
  free(S.v); free(T.v); free(M.v);
  return oom ? -1 : mults;
}

/* ---------------------------------------------------------------- sampled Dot2 */

/* TwoSum (Knuth): a + b = s + e exactly. */
static void two_sum(double a, double b, double* s, double* e) {
  double x = a + b, z = x - a;
  *s = x;
  *e = (a - (x - z)) + (b - z);
}

/* TwoProduct via a fused multiply-add: a*b = p + e exactly.  The compiler must not
 * contract or reorder these lines (the file is built with -ffp-contract=off). */
static void two_prod(double a, double b, double* p, double* e) {
  double x = a * b;
  *p = x;
  *e = __builtin_fma(a, b, -x);
}

/* For t = 0..count-1: out[t] = C0[rows[t]][cols[t]] + sum_p A[rows[t]][p] B[p][cols[t]],
 * the sum and the final addition carried in Dot2's (value, error) pair. */
void oracle_gemm_sampled(int64_t k, const double* A, int64_t lda,
                         const double* B, int64_t ldb,
                         const double* C0, int64_t ldc,
                         const int64_t* rows, const int64_t* cols, int64_t count,
                         double* out) {
  for (int64_t t = 0; t < count; ++t) {
    const int64_t i = rows[t], j = cols[t];
    double s = C0 ? C0[i * ldc + j] : 0.0, c = 0.0;
    for (int64_t p = 0; p < k; ++p) {
      double h, r, q;
      two_prod(A[i * lda + p], B[p * ldb + j], &h, &r);
      two_sum(s, h, &s, &q);
      c += q + r;
    }
    out[t] = s + c;
  }
}

/* ---------------------------------------------------------------- sampled Strassen */

/* Figure 1 once more, as data, for the entry-by-entry recursion below: for each product
 * M0..M6 its A terms, its B terms (block row, block column, sign; the first term's sign
 * is always +) and its C targets.  The rows and term orders are those of the
 * statements in oracle_strassen, so that every operand sum is formed the same way. */
typedef struct { int n; int bi[2], bj[2]; double sg[2]; } fig1_terms;
static const fig1_terms kFig1A[7] = {
  {2, {0, 1}, {0, 1}, {+1, +1}}, {2, {1, 1}, {0, 1}, {+1, +1}}, {1, {0, 0}, {0, 0}, {+1, 0}},
  {1, {1, 0}, {1, 0}, {+1, 0}},  {2, {0, 0}, {0, 1}, {+1, +1}}, {2, {1, 0}, {0, 0}, {+1, -1}},
  {2, {0, 1}, {1, 1}, {+1, -1}}};
static const fig1_terms kFig1B[7] = {
  {2, {0, 1}, {0, 1}, {+1, +1}}, {1, {0, 0}, {0, 0}, {+1, 0}},  {2, {0, 1}, {1, 1}, {+1, -1}},
  {2, {1, 0}, {0, 0}, {+1, -1}}, {1, {1, 0}, {1, 0}, {+1, 0}},  {2, {0, 0}, {0, 1}, {+1, +1}},
  {2, {1, 1}, {0, 1}, {+1, +1}}};
static const fig1_terms kFig1C[7] = {
  {2, {0, 1}, {0, 1}, {+1, +1}}, {2, {1, 1}, {0, 1}, {+1, -1}}, {2, {0, 1}, {1, 1}, {+1, +1}},
  {2, {0, 1}, {0, 0}, {+1, +1}}, {2, {0, 0}, {1, 0}, {+1, -1}}, {1, {1, 0}, {1, 0}, {+1, 0}},
  {1, {0, 0}, {0, 0}, {+1, 0}}};

/* A matrix that exists only as a recipe: either stored (element (r, c) at
 * X[r * rs + c * cs]) or the signed sum of quadrants of a parent, each quadrant
 * zero-padded past the parent's edge exactly as quad_load pads it. */
typedef struct vmat {
  const struct vmat* parent;
  int64_t rows, cols;
  const double* X; int64_t rs, cs;          /* stored */
  int n; int qi[2], qj[2]; double sg[2];   /* sum of parent quadrants */
} vmat;

/* out[0..cols) = row r of v (r < v->rows); returns 0, or -1 if out of memory. */
static int vmat_row(const vmat* v, int64_t r, double* out) {
  if (!v->parent) {
    for (int64_t c = 0; c < v->cols; ++c) out[c] = v->X[r * v->rs + c * v->cs];
    return 0;
  }
  const vmat* p = v->parent;
  double* buf = (double*)malloc(sizeof(double) * (size_t)(p->cols > 0 ? p->cols : 1));
  if (!buf) return -1;
  for (int t = 0; t < v->n; ++t) {
    const int64_t pr = v->qi[t] * v->rows + r;  /* the parent's row of this quadrant row */
    if (pr < p->rows) {
      if (vmat_row(p, pr, buf) < 0) { free(buf); return -1; }
    }
    for (int64_t c = 0; c < v->cols; ++c) {
      const int64_t pc = v->qj[t] * v->cols + c;
      const double x = (pr < p->rows && pc < p->cols) ? buf[pc] : 0.0;
      /* blk_copy for the first term, blk_add's x + s*y for the second */
      out[c] = (t == 0) ? x : out[c] + v->sg[t] * x;
    }
  }
  free(buf);
  return 0;
}

/* Entry (i, j) of c0 + (levels-level textbook Strassen of a (m x k) and bt^T, where bt
 * holds B transposed (n x k)), with the operations of oracle_strassen in its order:
 * per product the operand sums, the product recursively into a zeroed M, then
 * C += sign * M for the product's target quadrant; at the leaves the classical sum
 * over p in ascending order, then one addition into the target.  Returns 0 or -1. */
static int strassen_entry(int levels, const vmat* a, const vmat* bt, int64_t i, int64_t j, double c0,
                          double* out) {
  const int64_t m = a->rows, n = bt->rows, k = a->cols;
  if (levels <= 0) {
    double* ra = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    double* rb = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    if (!ra || !rb || vmat_row(a, i, ra) < 0 || vmat_row(bt, j, rb) < 0) { free(ra); free(rb); return -1; }
    double s = 0.0;
    for (int64_t p = 0; p < k; ++p) s += ra[p] * rb[p];
    free(ra); free(rb);
    *out = c0 + s;
    return 0;
  }
  const int64_t hm = (m + 1) / 2, hn = (n + 1) / 2, hk = (k + 1) / 2;
  const int qi = (int)(i / hm), qj = (int)(j / hn);
  const int64_t li = i - qi * hm, lj = j - qj * hn;
  double c = c0;
  for (int r = 0; r < 7; ++r) {
    double g = 0.0;
    for (int t = 0; t < kFig1C[r].n; ++t)
      if (kFig1C[r].bi[t] == qi && kFig1C[r].bj[t] == qj) g = kFig1C[r].sg[t];
    if (g == 0.0) continue;
    vmat sa, sb;
    memset(&sa, 0, sizeof(sa)); memset(&sb, 0, sizeof(sb));
    sa.parent = a; sa.rows = hm; sa.cols = hk; sa.n = kFig1A[r].n;
    sb.parent = bt; sb.rows = hn; sb.cols = hk; sb.n = kFig1B[r].n;
    for (int t = 0; t < 2; ++t) {
      sa.qi[t] = kFig1A[r].bi[t]; sa.qj[t] = kFig1A[r].bj[t]; sa.sg[t] = kFig1A[r].sg[t];
      /* quadrant (bi, bj) of B is quadrant (bj, bi) of its transpose */
      sb.qi[t] = kFig1B[r].bj[t]; sb.qj[t] = kFig1B[r].bi[t]; sb.sg[t] = kFig1B[r].sg[t];
    }
    double M;
    if (strassen_entry(levels - 1, &sa, &sb, li, lj, 0.0, &M) < 0) return -1;
    c += g * M;
  }
  *out = c;
  return 0;
}

/* For t = 0..count-1: out[t] = entry (rows[t], cols[t]) of what oracle_strassen(levels,
 * m, n, k, A, lda, B, ldb, C) leaves in C when C starts as C0 (NULL: zeros), bit for
 * bit.  B is passed transposed: Bt is n x k with row stride ldbt.  Returns 0 or -1. */
int oracle_strassen_sampled(int levels, int64_t m, int64_t n, int64_t k,
                            const double* A, int64_t lda,
                            const double* Bt, int64_t ldbt,
                            const double* C0, int64_t ldc,
                            const int64_t* rows, const int64_t* cols, int64_t count,
                            double* out) {
  vmat a, bt;
  memset(&a, 0, sizeof(a)); memset(&bt, 0, sizeof(bt));
  a.rows = m; a.cols = k; a.X = A; a.rs = lda; a.cs = 1;
  bt.rows = n; bt.cols = k; bt.X = Bt; bt.rs = ldbt; bt.cs = 1;
  for (int64_t t = 0; t < count; ++t) {
    const int64_t i = rows[t], j = cols[t];
    const double c0 = C0 ? C0[i * ldc + j] : 0.0;
    if (k <= 0) { out[t] = c0; continue; }
    if (strassen_entry(levels, &a, &bt, i, j, c0, &out[t]) < 0) return -1;
  }
  return 0;
}
