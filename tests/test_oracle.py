"""Pins of the CPU oracle to facts the paper and the mathematics fix (no GPU).

Each test ties the oracle to something other than itself: exact integer products
computed by brute force in Python integers, the figures of the paper transcribed in
``tests/golden/``, multiplication counts (Section 3.1-3.2), cost counts of the model
(Section 4.2), and exactly known sums for the compensated dot product.
"""
import fractions
import os

import numpy as np
import pytest

import oracle
from oracle import tables
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute(A, B, C):
    """C + A B in exact Python integers (inputs must be integer-valued)."""
    m, k = A.shape
    n = B.shape[1]
    Ai = [[int(A[i, p]) for p in range(k)] for i in range(m)]
    Bi = [[int(B[p, j]) for j in range(n)] for p in range(k)]
    out = np.empty((m, n))
    for i in range(m):
        for j in range(n):
            out[i, j] = int(C[i, j]) + sum(Ai[i][p] * Bi[p][j] for p in range(k))
    return out


def parse_terms(field, signed):
    toks = field.split()
    out = []
    for t in toks:
        if signed:
            s = -1 if t[0] == "-" else 1
            t = t[1:]
        else:
            s = 1
        out.append((int(t[0]), int(t[1]), s))
    return tuple(out)


def load_fig(name, signed_operands):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            r, a, b, c = [f.strip() for f in line.split("|")]
            rows.append((int(r), parse_terms(a, signed_operands), parse_terms(b, signed_operands),
                         parse_terms(c, True)))
    return rows


# ---------------------------------------------------------------- classical definition

@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (3, 5, 7), (8, 8, 8), (13, 6, 11)])
def test_gemm_matches_bruteforce_integers(m, n, k):
    A, B, C = W.integer(m, k, 1), W.integer(k, n, 2), W.integer(m, n, 3)
    out = C.copy()
    assert oracle.gemm(A, B, out) == m * n * k
    assert np.array_equal(out, brute(A, B, C))


def test_gemm_respects_leading_dimensions():
    A = W.integer(9, 7, 4, ld=11)
    B = W.integer(7, 5, 5, ld=8)
    buf = np.full((9, 13), 123.0)
    C = buf[:, :5]
    C[:] = 0
    oracle.gemm(A, B, C)
    assert np.array_equal(C, brute(np.ascontiguousarray(A), np.ascontiguousarray(B), np.zeros((9, 5))))
    assert np.all(buf[:, 5:] == 123.0)  # padding of C untouched


def test_gemm_identity_and_permutation():
    B = W.uniform(6, 9, 7)
    C = np.zeros((6, 9))
    oracle.gemm(np.eye(6), B, C)
    assert np.array_equal(C, B)
    P = np.eye(6)[[3, 0, 5, 1, 4, 2]]
    C = np.zeros((6, 9))
    oracle.gemm(P, B, C)
    assert np.array_equal(C, B[[3, 0, 5, 1, 4, 2]])


def test_gemm_float_close_to_numpy():
    A, B = W.uniform(40, 50, 8), W.uniform(50, 30, 9)
    C = np.zeros((40, 30))
    oracle.gemm(A, B, C)
    assert np.max(np.abs(C - A @ B)) < 1e-13


# ---------------------------------------------------------------- textbook Strassen

@pytest.mark.parametrize("levels", [1, 2, 3])
@pytest.mark.parametrize("m,n,k", [(16, 16, 16), (13, 7, 11), (1, 1, 1), (2, 3, 5), (17, 16, 15)])
def test_strassen_exact_on_integers(levels, m, n, k):
    A, B, C = W.integer(m, k, 10 + levels), W.integer(k, n, 20 + levels), W.integer(m, n, 30)
    out = C.copy()
    oracle.strassen(A, B, out, levels)
    assert np.array_equal(out, brute(A, B, C))


def test_strassen_config_16x16_integer_case():
    """The 16x16 integer-valued case with entries in {-4..4}."""
    A, B = W.integer(16, 16, 0), W.integer(16, 16, 1)
    ref = brute(A, B, np.zeros((16, 16)))
    for L in (0, 1, 2):
        out = np.zeros((16, 16))
        oracle.strassen(A, B, out, L)
        assert np.array_equal(out, ref)


@pytest.mark.parametrize("d", [3, 5])
def test_strassen_multiplication_counts(d):
    """7^L products of (n/2^L)^3 multiplies against 8^L for the block product of
    Section 2.3 (Sections 3.1-3.2: cost (7/8)^L 2n^3)."""
    n = 2 ** d
    A, B = W.uniform(n, n, 1), W.uniform(n, n, 2)
    for L in range(0, 4):
        mults = oracle.strassen(A, B, np.zeros((n, n)), L)
        assert mults == 7 ** L * (n // 2 ** L) ** 3
        assert mults * 8 ** L == 7 ** L * n ** 3


def test_strassen_counts_with_padding():
    # 13 x 7 x 11 with one level: padded halves 7, 4, 6
    mults = oracle.strassen(W.uniform(13, 11, 1), W.uniform(11, 7, 2), np.zeros((13, 7)), 1)
    assert mults == 7 * 7 * 4 * 6


def test_strassen_identity_with_integer_partner():
    B = W.integer(12, 10, 3)
    for L in (1, 2):
        out = np.zeros((12, 10))
        oracle.strassen(np.eye(12), B, out, L)
        assert np.array_equal(out, B)


def test_two_levels_equal_one_level_twice():
    """Section 3.2: a product of one-level Strassen computed by one-level Strassen is
    two-level Strassen; on integers both forms are exact, so they agree bit for bit,
    and the flat two-level table of Eq. 3 gives the same result."""
    A, B = W.integer(20, 24, 5), W.integer(24, 18, 6)
    two = np.zeros((20, 18))
    oracle.strassen(A, B, two, 2)
    flat = tables.apply_table(A, B, np.zeros((20, 18)), 2)
    assert np.array_equal(two, flat)
    assert np.array_equal(two, brute(A, B, np.zeros((20, 18))))


def test_three_levels_recursive_flat_and_bruteforce_agree():
    """Sections 3.5-3.6 one level further: recursive three-level Strassen, the flat
    343-product table of Eq. 4 and brute force agree bit for bit on integers, on a
    ragged shape whose blocks are padded at every level."""
    A, B, C = W.integer(37, 29, 15), W.integer(29, 41, 16), W.integer(37, 41, 17)
    rec = C.copy()
    oracle.strassen(A, B, rec, 3)
    flat = tables.apply_table(A, B, C, 3)
    ref = brute(A, B, C)
    assert np.array_equal(rec, ref)
    assert np.array_equal(flat, ref)


def test_three_level_table_is_the_associative_kronecker_cube():
    """The three-level table built as (two-level) x (Figure 1) equals the one built as
    (Figure 1) x (two-level) with product index 49 a + b and block index 4 outer + inner:
    the Kronecker product is associative, so both orders name the same 343 products."""
    def kron(outer, inner, w):
        return tuple((w * oi + ii, w * oj + ij, os * s) for (oi, oj, os) in outer for (ii, ij, s) in inner)
    other = [(kron(fa, ta, 4), kron(fb, tb, 4), kron(fc, tc, 4))
             for (fa, fb, fc) in tables.FIG1 for (ta, tb, tc) in tables.table(2)]
    assert other == tables.table(3)
    c3 = tables.counts(3)
    assert c3["products"] == 343 and c3["a_terms"] == 12 ** 3 and c3["c_updates"] == 12 ** 3


@pytest.mark.parametrize("levels", [0, 1, 2, 3])
@pytest.mark.parametrize("m,n,k", [(37, 41, 29), (1, 9, 4), (64, 64, 64), (100, 77, 130)])
def test_strassen_sampled_equals_full_recursion(levels, m, n, k):
    """The entry-by-entry textbook Strassen repeats the full recursion's operations in
    its order: on float inputs (where every rounding shows) and ragged shapes (padding
    at every level) every entry agrees bit for bit, with and without C0."""
    A, B, C = W.uniform(m, k, 1), W.uniform(k, n, 2), W.uniform(m, n, 3)
    rows, cols = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    for C0 in (C, None):
        full = np.zeros((m, n)) if C0 is None else C0.copy()
        oracle.strassen(A, B, full, levels)
        got = oracle.strassen_sampled(A, B, C0, rows.ravel(), cols.ravel(), levels).reshape(m, n)
        assert np.array_equal(got, full)


def test_timing_build_computes_the_same_entries():
    """The OpenMP timing build splits rows over threads but computes every entry with
    the same operations: bit for bit the result of the plain build."""
    A, B, C = W.uniform(130, 97, 1), W.uniform(97, 111, 2), W.uniform(130, 111, 3)
    for L in (0, 1, 2):
        ref = C.copy()
        oracle.strassen(A, B, ref, L)
        for threads in (1, 3):
            got = C.copy()
            oracle.strassen_timed(A, B, got, L, threads)
            assert np.array_equal(got, ref)
    assert oracle.host_cores() >= 1


def test_strassen_sampled_exact_on_integers_and_strided_operands():
    A = W.integer(23, 19, 4, ld=25)
    B = W.integer(19, 17, 5, ld=20)
    C = W.integer(23, 17, 6)
    ref = brute(np.ascontiguousarray(A), np.ascontiguousarray(B), C)
    rows, cols = W.sample_indices(23, 17, 50, 3)
    for L in (1, 2, 3):
        assert np.array_equal(oracle.strassen_sampled(A, B, C, rows, cols, L), ref[rows, cols])


@pytest.mark.parametrize("levels,tol", [(1, 1e-13), (2, 1e-12), (3, 1e-12)])
def test_strassen_float_error_scale(levels, tol):
    n = 192
    A, B = W.uniform(n, n, 11), W.uniform(n, n, 12)
    out = np.zeros((n, n))
    oracle.strassen(A, B, out, levels)
    rows, cols = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ref = oracle.gemm_sampled(A, B, None, rows.ravel(), cols.ravel()).reshape(n, n)
    assert oracle.max_rel_err(out, ref, A, B) < tol


# ---------------------------------------------------------------- tables vs. the figures

def test_fig1_table_matches_print():
    printed = load_fig("fig1_one_level.txt", signed_operands=True)
    assert len(printed) == 7
    for (r, a, b, c), (ta, tb, tc) in zip(printed, tables.FIG1):
        assert (a, b, c) == (ta, tb, tc), f"M{r}"


def test_kronecker_table_matches_fig2_terms_and_c_signs():
    printed = load_fig("fig2_two_level.txt", signed_operands=False)
    assert len(printed) == 49
    gen = tables.table(2)
    for (r, a, b, c), (ga, gb, gc) in zip(printed, gen):
        assert sorted((i, j) for i, j, _ in a) == sorted((i, j) for i, j, _ in ga), f"A terms of M{r}"
        assert sorted((i, j) for i, j, _ in b) == sorted((i, j) for i, j, _ in gb), f"B terms of M{r}"
        assert sorted(c) == sorted(gc), f"C updates of M{r}"


def test_fig2_operand_signs_as_printed_do_not_compute_ab():
    """With every operand sign '+', as Figure 2 prints them, the products do not give
    A*B; the signs must come from the Kronecker square of Figure 1."""
    printed = load_fig("fig2_two_level.txt", signed_operands=False)
    tab = [(a, b, c) for (_, a, b, c) in printed]
    A, B = W.integer(16, 16, 0), W.integer(16, 16, 1)
    got = tables.apply_table(A, B, np.zeros((16, 16)), 2, tab)
    assert not np.array_equal(got, A @ B)


@pytest.mark.parametrize("levels", [0, 1, 2, 3])
def test_table_computes_ab_exactly(levels):
    A, B, C = W.integer(19, 23, 7), W.integer(23, 17, 8), W.integer(19, 17, 9)
    got = tables.apply_table(A, B, C, levels)
    assert np.array_equal(got, brute(A, B, C))


def test_table_sign_mutation_is_detected():
    """A single flipped sign anywhere in Figure 1 breaks A*B on integers."""
    A, B = W.integer(8, 8, 3), W.integer(8, 8, 4)
    ref = A @ B
    for r in range(7):
        for part in range(3):
            tab = [list(p) for p in tables.FIG1]
            terms = list(tab[r][part])
            i, j, s = terms[0]
            terms[0] = (i, j, -s)
            tab[r][part] = tuple(terms)
            got = tables.apply_table(A, B, np.zeros((8, 8)), 1, [tuple(p) for p in tab])
            assert not np.array_equal(got, ref), (r, part)


def test_cost_counts_match_model_table():
    """Section 4.2: one level has 7 products, 5 extra additions of A and of B blocks
    and 12 additions into C; two levels 49 products and 95 extra additions (printed),
    and 144 C updates (the model prints 154 for two levels: see the design notes)."""
    c1, c2 = tables.counts(1), tables.counts(2)
    printed = {}
    with open(os.path.join(GOLDEN, "model_counts.txt")) as fh:
        for line in fh:
            f = line.split()
            if f and f[0] == "arith":
                printed[int(f[1])] = tuple(int(x) for x in f[2:])
    assert (c1["products"], c1["a_adds"], c1["b_adds"], c1["c_updates"]) == printed[1]
    assert (c2["products"], c2["a_adds"], c2["b_adds"]) == printed[2][:3]
    assert c2["c_updates"] == 144 and printed[2][3] == 154
    assert c1["a_terms"] == 12 and c2["a_terms"] == 144


# ---------------------------------------------------------------- compensated sampled entries

def test_dot2_recovers_cancelled_sum():
    A = np.array([[1e16, 1.0, -1e16, 3.0]])
    B = np.array([[1.0], [1.0], [1.0], [1.0]])
    got = oracle.gemm_sampled(A, B, None, np.array([0]), np.array([0]))
    assert got[0] == 4.0
    naive = np.zeros((1, 1))
    oracle.gemm(A, B, naive)
    assert naive[0, 0] != 4.0


def test_dot2_against_exact_rationals():
    A, B, C0 = W.uniform(5, 300, 21), W.uniform(300, 4, 22), W.uniform(5, 4, 23)
    rows, cols = np.repeat(np.arange(5), 4), np.tile(np.arange(4), 5)
    got = oracle.gemm_sampled(A, B, C0, rows, cols)
    for t, (i, j) in enumerate(zip(rows, cols)):
        exact = fractions.Fraction(C0[i, j]) + sum(fractions.Fraction(A[i, p]) * fractions.Fraction(B[p, j])
                                                   for p in range(300))
        err = abs(fractions.Fraction(got[t]) - exact)
        assert err <= abs(exact) * fractions.Fraction(2, 2 ** 53) + fractions.Fraction(1, 2 ** 100)


def test_max_rel_err_definition():
    A, B = np.array([[2.0, -4.0]]), np.array([[0.5], [3.0]])
    assert oracle.max_rel_err(np.array([[1.0]]), np.array([[0.0]]), A, B) == 1.0 / 12.0


# ---------------------------------------------------------------- BLAS semantics (Section 2.2)

@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_dgemm_definition_on_integers(ta, tb):
    """alpha op(A) op(B) + beta C against brute-force triple loops on integers."""
    m, n, k = 7, 5, 6
    A = W.integer(k, m, 1) if ta else W.integer(m, k, 1)
    B = W.integer(n, k, 2) if tb else W.integer(k, n, 2)
    C = W.integer(m, n, 3)
    got = oracle.dgemm(ta, tb, 3.0, A, B, -2.0, C)
    for i in range(m):
        for j in range(n):
            acc = 0.0
            for p in range(k):
                a = A[p, i] if ta else A[i, p]
                b = B[j, p] if tb else B[p, j]
                acc += a * b
            assert got[i, j] == 3.0 * acc - 2.0 * C[i, j]


def test_dgemm_reduces_to_gemm_and_respects_beta_zero():
    A, B, C = W.integer(9, 4, 4), W.integer(4, 8, 5), W.integer(9, 8, 6)
    ref = C.copy()
    oracle.gemm(A, B, ref)
    assert np.array_equal(oracle.dgemm(0, 0, 1.0, A, B, 1.0, C), ref)
    Cnan = np.full((9, 8), np.nan)
    assert np.array_equal(oracle.dgemm(0, 0, 1.0, A, B, 0.0, Cnan), A @ B)
    assert np.array_equal(oracle.dgemm(1, 1, 2.0, A.T.copy(), B.T.copy(), 0.0, Cnan), 2 * (A @ B))
    assert np.array_equal(oracle.dgemm(0, 0, 0.0, A, B, 0.5, C), 0.5 * C)


# ---------------------------------------------------------------- symmetric rank-k update

@pytest.mark.parametrize("uplo", [0, 1])
@pytest.mark.parametrize("trans", [0, 1])
def test_dsyrk_definition_on_integers(uplo, trans):
    """alpha op(A) op(A)^T + beta C on one triangle, against brute force in exact
    integers; the other triangle is returned untouched (NaN stays NaN)."""
    n, k = 11, 7
    A = W.integer(k, n, 3) if trans else W.integer(n, k, 3)
    C = W.integer(n, n, 4)
    i, j = np.indices((n, n))
    tri = (j <= i) if uplo == 0 else (j >= i)
    C[~tri] = np.nan
    Aop = np.ascontiguousarray(A.T if trans else A)
    P = brute(Aop, np.ascontiguousarray(Aop.T), np.zeros((n, n)))
    out = oracle.dsyrk(uplo, trans, 2.0, A, -3.0, C)
    assert np.array_equal(out[tri], (2.0 * P - 3.0 * C)[tri])
    assert np.all(np.isnan(out[~tri]))


def test_dsyrk_triangles_are_transposes_and_beta_zero_ignores_c():
    n, k = 9, 13
    A = W.integer(n, k, 5)
    C = W.integer(n, n, 6)
    C = C + C.T  # symmetric
    lo = oracle.dsyrk(0, 0, 1.0, A, 1.0, C)
    up = oracle.dsyrk(1, 0, 1.0, A, 1.0, C)
    assert np.array_equal(np.tril(lo), np.tril(up.T))
    Cn = np.full((n, n), np.nan)
    z = oracle.dsyrk(0, 0, 1.0, A, 0.0, Cn)
    assert np.array_equal(np.tril(z), np.tril(brute(A, np.ascontiguousarray(A.T), np.zeros((n, n)))))
    # k = 0: only the scaling by beta
    e = oracle.dsyrk(1, 0, 5.0, np.zeros((n, 0)), 2.0, C)
    assert np.array_equal(np.triu(e), np.triu(2.0 * C))
