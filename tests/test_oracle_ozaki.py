"""Pins of the split-precision (Ozaki-style) oracle: exact digit splitting, digit
bounds, exact integer slice products, exactness on integer and single-binade inputs,
the FP64-level error on random inputs, and its use under Strassen (no GPU)."""

import numpy as np
import pytest

import oracle
from oracle import ozaki
import workloads as W


BITS, S0 = ozaki.B_BITS, ozaki.S_DIGITS


def test_scheme_parameters():
    """Digits of 8 bits, seven per operand: 56 bits, and |d| <= 128 is exact in BF16
    (8 significant bits) while a digit product (<= 2^14) is exact in FP32."""
    assert (BITS, S0) == (8, 7)
    assert float(np.float32(2.0 ** 14)) == 2.0 ** 14


@pytest.mark.parametrize("b,S_list", [(8, (3, 5, 7)), (7, (3, 8))])
def test_split_reconstructs_exactly_and_digits_are_bounded(b, S_list):
    U = np.ldexp(W.uniform(40, 50, 1), -1) * 0.999  # entries in (-1/2, 1/2)
    for S in S_list:
        D = ozaki.split(U, S, b)
        assert np.all(np.abs(D) <= 2 ** (b - 1)) and np.all(D == np.rint(D))
        N = sum(D[s].astype(np.int64) << (b * (S - 1 - s)) for s in range(S))
        assert np.array_equal(N, np.rint(np.ldexp(U, b * S)).astype(np.int64))
        # the digits carry U to within half a unit of the last digit
        rebuilt = np.ldexp(N.astype(np.float64), -b * S)
        assert np.all(np.abs(rebuilt - U) <= 2.0 ** (-b * S - 1))


def test_split_extreme_digits():
    # the largest magnitude just below 1/2, a tie at every digit, and a negative tie
    U = np.array([[0.5 - 2.0 ** -56, 2.0 ** -9 * 0.5, -(2.0 ** -9) * 0.5, 0.0, -0.5 + 2.0 ** -56]])
    D = ozaki.split(U, S0)
    assert np.all(np.abs(D) <= 128)
    assert np.max(np.abs(D)) == 128      # the bound is reached
    N = sum(D[s].astype(np.int64) << (BITS * (S0 - 1 - s)) for s in range(S0))
    assert np.array_equal(N, np.rint(np.ldexp(U, 56)).astype(np.int64))


def test_seven_digits_cover_one_binade_exactly():
    """Entries in +-[1/4, 1/2) have 53-bit mantissas ending at 2^-54: seven 8-bit
    digits (56 bits) represent them with zero remainder."""
    g = np.random.Generator(np.random.Philox(5))
    U = np.copysign(g.uniform(0.25, 0.5, size=(30, 30)), g.uniform(-1, 1, size=(30, 30)))
    D = ozaki.split(U, S0)
    assert np.array_equal(sum(D[s] * 2.0 ** (-BITS * (s + 1)) for s in range(S0)), U)


def test_scale_exponents():
    X = np.array([[0.49, -0.1], [0.5, 0.0], [0.0, 0.0], [-3.0, 1.0]])
    e = ozaki.scale_exponents_rows(X)
    assert list(e) == [0, 1, 0, 3]
    for i in (0, 1, 3):
        assert np.max(np.abs(X[i])) < 2.0 ** (e[i] - 1) and np.max(np.abs(X[i])) >= 2.0 ** (e[i] - 2)


def test_group_products_are_exact_integers():
    g = np.random.Generator(np.random.Philox(9))
    DX = g.integers(-128, 129, size=(3, 4, 6)).astype(np.float64)
    DV = g.integers(-128, 129, size=(3, 6, 5)).astype(np.float64)
    G = ozaki.slice_product_groups(DX, DV)
    assert sorted(G) == [2, 3, 4]
    for w in (2, 3, 4):
        for i in range(4):
            for j in range(5):
                ref = sum(int(DX[s - 1, i, p]) * int(DV[w - s - 1, p, j])
                          for s in range(1, w) if w - s <= 3 for p in range(6))
                assert G[w][i, j] == ref


@pytest.mark.parametrize("m,n,k", [(8, 9, 10), (33, 17, 65)])
def test_integer_inputs_give_the_exact_product(m, n, k):
    A, B = W.integer(m, k, 1, lo=-60, hi=60), W.integer(k, n, 2, lo=-60, hi=60)
    assert np.array_equal(ozaki.product(A, B), A @ B)


def test_float_error_is_at_fp64_level():
    m, n, k = 24, 20, 300
    A, B = W.uniform(m, k, 3), W.uniform(k, n, 4)
    got = ozaki.product(A, B)
    rows, cols = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    exact = oracle.gemm_sampled(A, B, None, rows.ravel(), cols.ravel()).reshape(m, n)
    bound = (k + 1) * 2.0 ** -53 * (np.abs(A) @ np.abs(B))  # the classical FP64 bound
    assert np.all(np.abs(got - exact) <= bound)


def test_fewer_slices_lose_accuracy_monotonically():
    A, B = W.uniform(16, 64, 5), W.uniform(64, 16, 6)
    ref = A @ B
    errs = [np.max(np.abs(ozaki.product(A, B, S=s) - ref)) for s in (2, 3, 5)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] > 1e-6


@pytest.mark.parametrize("sigma", [0, 4, 10])
def test_spread_exponents_error_within_scaled_bound(sigma):
    """Error bound of the scheme: with S = 7 digits of 8 bits the dropped digit tails
    and slice pairs contribute at most about k 2^(e_i + f_j) 2^-55, and the one
    rounding of the recombination half an ulp of the result; 2^(e_i + f_j) k 2^-50
    covers both."""
    k = 200
    A, B = W.scaled(20, k, 7, sigma), W.scaled(k, 18, 8, sigma)
    got = ozaki.product(A, B)
    rows, cols = np.meshgrid(np.arange(20), np.arange(18), indexing="ij")
    exact = oracle.gemm_sampled(A, B, None, rows.ravel(), cols.ravel()).reshape(20, 18)
    e, f = ozaki.scale_exponents_rows(A), ozaki.scale_exponents_rows(B.T)
    bound = np.ldexp(np.full((20, 18), k * 2.0 ** -50), (e[:, None] + f[None, :]).astype(np.int64))
    assert np.all(np.abs(got - exact) <= bound)
    # and a dropped pair group would break it
    S = S0
    DX = ozaki.split(np.ldexp(A, -e[:, None]), S)
    DV = ozaki.split(np.ldexp(B, -f[None, :]), S)
    G = ozaki.slice_product_groups(DX, DV)
    G[3] = np.zeros_like(G[3])
    broken = ozaki.recombine(G, e, f, S)
    assert not np.all(np.abs(broken - exact) <= bound)


@pytest.mark.parametrize("levels", [0, 1, 2, 3])
def test_strassen_with_split_products_exact_on_integers(levels):
    A, B, C = W.integer(21, 19, 1), W.integer(19, 23, 2), W.integer(21, 23, 3)
    got = ozaki.gemm(A, B, C, levels)
    assert np.array_equal(got, C + A @ B)


def test_identity_and_powers_of_two():
    X = np.ldexp(np.ones((6, 6)), np.arange(36).reshape(6, 6) % 7 - 3)
    assert np.array_equal(ozaki.product(np.eye(6), X), X)
    assert np.array_equal(ozaki.product(X, np.eye(6)), X)


def test_recombination_is_the_correctly_rounded_exact_sum():
    """Step 4 against exact rational arithmetic: M = RN(sum_w G_w 2^(-bw) 2^(e+f))."""
    import fractions
    A, B = W.uniform(5, 40, 11), W.scaled(40, 4, 12, 3)
    S = S0
    e, f = ozaki.scale_exponents_rows(A), ozaki.scale_exponents_rows(B.T)
    DX = ozaki.split(np.ldexp(A, -e[:, None]), S)
    DV = ozaki.split(np.ldexp(B, -f[None, :]), S)
    G = ozaki.slice_product_groups(DX, DV)
    M = ozaki.recombine(G, e, f, S)
    for i in range(5):
        for j in range(4):
            exact = sum(fractions.Fraction(int(G[w][i, j])) * fractions.Fraction(2) ** (-BITS * w) for w in G)
            exact *= fractions.Fraction(2) ** int(e[i] + f[j])
            assert M[i, j] == float(exact)
