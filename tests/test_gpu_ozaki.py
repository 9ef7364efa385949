"""GPU parity of the split-precision path (dtype STRASSEN_F64_OZ_BF16, tensor-core BF16
slice products) against the oracle of the same scheme, through the C ABI.

The slice products are exact integers on both sides and the recombination is one
correctly rounded conversion followed by the C additions in product order, so the GPU
result must equal the oracle bit for bit on any finite input.  Against the exact product
(the oracle's Dot2 entries) the error is held to the strict FP64 tolerance
max|C - C_exact| / (max|A| max|B|) <= 1e-13 (one level and classical slices) or 1e-12
(two levels) for sigma = 0; the benchmark states it per sigma.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import ozaki
import paper_1605_01078_gb300 as sg
import workloads as W

pytestmark = pytest.mark.gpu

OZ = "oz_bf16"
TOL = {0: 1e-13, 1: 1e-13, 2: 1e-12}


def effective_levels(levels, m, n, k):
    """The library clamps levels while 2^levels exceeds min(m, n, k)."""
    while levels > 0 and (1 << levels) > min(m, n, k):
        levels -= 1
    return levels


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run(A, B, C, levels):
    dC = dev(C)
    sg.gemm(dev(A), dev(B), dC, levels=levels, variant="ABC", dtype=OZ)
    torch.cuda.synchronize()
    assert sg.strassen_device_status(0) == 0
    return dC.cpu().numpy()


@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("m,n,k", [(16, 16, 16), (130, 70, 150), (300, 260, 2100), (1, 1, 1), (5, 129, 3)])
def test_bit_exact_against_the_scheme_oracle(levels, m, n, k):
    A, B, C = W.uniform(m, k, 1), W.uniform(k, n, 2), W.uniform(m, n, 3)
    ref = ozaki.gemm(A, B, C, effective_levels(levels, m, n, k))
    got = run(A, B, C, levels)
    assert np.array_equal(got, ref), float(np.max(np.abs(got - ref)))


@pytest.mark.parametrize("levels", [0, 1])
def test_bit_exact_over_several_pair_tiles(levels):
    """Several 256 x 256 tiles of CTA pairs in both directions, with ragged last rows and
    columns (h_m = 700 >> levels, h_n = 600 >> levels)."""
    m, n, k = 700, 600, 520
    A, B, C = W.uniform(m, k, 21), W.uniform(k, n, 22), W.uniform(m, n, 23)
    assert np.array_equal(run(A, B, C, levels), ozaki.gemm(A, B, C, levels))


def test_concurrent_with_fp64_work_on_another_stream():
    """A split-precision call launched while a long FP64 product runs on another stream:
    its CTA pairs start as SMs free up, so some join the pacing count late; the result is
    still the scheme's, bit for bit, and the call reports no timeout."""
    m, n, k = 700, 600, 520
    A, B, C = W.uniform(m, k, 31), W.uniform(k, n, 32), W.uniform(m, n, 33)
    ref = ozaki.gemm(A, B, C, 1)
    big = [W.uniform_device(4096, 4096, s) for s in (34, 35, 36)]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    dA, dB, dC = dev(A), dev(B), dev(C)
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        sg.gemm(big[0], big[1], big[2], levels=2, stream=s1)
    with torch.cuda.stream(s2):
        sg.gemm(dA, dB, dC, levels=1, variant="ABC", dtype=OZ, stream=s2)
    torch.cuda.synchronize()
    assert sg.strassen_device_status(0) == 0
    assert np.array_equal(dC.cpu().numpy(), ref)


@pytest.mark.parametrize("sigma", [4, 10])
def test_bit_exact_with_spread_exponents(sigma):
    A, B, C = W.scaled(200, 300, 4, sigma), W.scaled(300, 150, 5, sigma), W.scaled(200, 150, 6, sigma)
    for levels in (0, 1):
        assert np.array_equal(run(A, B, C, levels), ozaki.gemm(A, B, C, levels))


def test_three_levels_bit_exact_against_the_scheme_oracle():
    A, B, C = W.uniform(130, 150, 1), W.uniform(150, 70, 2), W.uniform(130, 70, 3)
    assert np.array_equal(run(A, B, C, 3), ozaki.gemm(A, B, C, 3))


def test_integer_inputs_exact():
    A, B, C = W.integer(100, 90, 7), W.integer(90, 80, 8), W.integer(100, 80, 9)
    for levels in (0, 1, 2, 3):
        assert np.array_equal(run(A, B, C, levels), C + A @ B)


@pytest.mark.parametrize("levels", [0, 1, 2])
def test_fp64_tolerance_config_1024(levels):
    n = 1024
    A, B, C = W.uniform(n, n, 0), W.uniform(n, n, 1), np.zeros((n, n))
    got = run(A, B, C, levels)
    rows, cols = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    exact = oracle.gemm_sampled(A, B, None, rows.ravel(), cols.ravel()).reshape(n, n)
    assert oracle.max_rel_err(got, exact, A, B) <= TOL[levels]


def test_full_size_classical_slices_bit_exact_on_sampled_entries():
    """8192^3 classical slices, many waves of CTA pairs: at level 0 an entry of the
    scheme depends only on its row of A and its column of B (their scales included), so
    the oracle's product of the sampled rows and columns gives those entries exactly."""
    n = 8192
    A, B, C = W.uniform(n, n, 110), W.uniform(n, n, 111), W.uniform(n, n, 112)
    got = run(A, B, C, 0)
    rows, cols = W.sample_indices(n, n, 256, 7)
    R, ri = np.unique(rows, return_inverse=True)
    Q, qi = np.unique(cols, return_inverse=True)
    M = ozaki.product(A[R], B[:, Q])
    assert np.array_equal(got[rows, cols], C[rows, cols] + M[ri, qi])


@pytest.mark.parametrize("levels", [0, 1, 2])
def test_full_size_sampled(levels):
    n = 8192
    A, B, C = W.uniform(n, n, 100), W.uniform(n, n, 101), W.uniform(n, n, 102)
    got = run(A, B, C, levels)
    rows, cols = W.sample_indices(n, n, 256, 3)
    ref = oracle.gemm_sampled(A, B, C, rows, cols)
    assert oracle.max_rel_err(got[rows, cols], ref, A, B) <= TOL[levels]


def test_int8_slices_not_built():
    A = dev(np.ones((4, 4)))
    C = dev(np.zeros((4, 4)))
    st = sg.strassen_gemm(4, 4, 4, A.data_ptr(), 4, A.data_ptr(), 4, C.data_ptr(), 4, 0, 0,
                          sg.STRASSEN_F64_OZ_INT8, 0)
    assert st == -5


@pytest.mark.parametrize("k", [512, 1024, 3000])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_extreme_digits_fill_the_exact_chunk_bound(k, sign):
    """Every entry 0.5 - 2^-54 (top digit 128): each full 1024-product FP32 chunk of the
    top-digit pair sums to exactly +-2^24 (k = 1024, 3000), every partial sum an
    integer within the FP32 exact range, the largest value the exactness argument
    allows; the result must still match the scheme bit for bit."""
    x = 0.5 - 2.0 ** -54
    A, B = np.full((64, k), x), np.full((k, 64), sign * x)
    C = np.zeros((64, 64))
    ref = ozaki.gemm(A, B, C, 0)
    assert np.array_equal(run(A, B, C, 0), ref)


def test_long_reduction_uses_several_k_segments():
    """k = 16448 needs two k segments (each keeps the int32 group sums below 2^31);
    the recombination adds them exactly."""
    A, B, C = W.uniform(70, 16448, 21), W.uniform(16448, 50, 22), W.uniform(70, 50, 23)
    assert np.array_equal(run(A, B, C, 0), ozaki.gemm(A, B, C, 0))


def test_stage_profile_times_a_normal_call():
    """strassen_profile_split_precision makes one ordinary split-precision call (the same
    C as strassen_gemm, bit for bit) and reports three positive stage times."""
    m, n, k = 700, 650, 900
    A, B, C = W.uniform(m, k, 5), W.uniform(k, n, 6), W.uniform(m, n, 7)
    for levels in (0, 1, 2):
        want = run(A, B, C, levels)
        dA, dB, dC = dev(A), dev(B), dev(C)
        ms = sg.strassen_profile_split_precision(m, n, k, dA.data_ptr(), k, dB.data_ptr(), n, dC.data_ptr(), n,
                                                 levels, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(dC.cpu().numpy(), want)
        assert len(ms) == 3 and all(t > 0 for t in ms)
    with pytest.raises(sg.StrassenError):
        sg.strassen_profile_split_precision(m, n, k, dA.data_ptr(), k, dB.data_ptr(), n, dC.data_ptr(), n, 4, 0)
