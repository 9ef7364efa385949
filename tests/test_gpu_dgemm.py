"""GPU parity of strassen_dgemm, C = alpha op(A) op(B) + beta C (the BLAS operation of
Section 2.2), against the oracle's definition: every transpose combination, level and
variant bit for bit on integer inputs with integer alpha and beta; a float case within
the tolerance; beta = 0 over NaN-filled C; alpha = 0; transposed operands with padded
leading dimensions; the split-precision dtype bit for bit against its scheme."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import ozaki
import paper_1605_01078_gb300 as sg
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 1e-13, 2: 1e-12, 3: 1e-12}


def dev(x, ld=None):
    rows, cols = x.shape
    if ld is None or ld == cols:
        return torch.from_numpy(np.ascontiguousarray(x)).cuda()
    buf = torch.full((rows, ld), float("nan"), dtype=torch.float64, device="cuda")
    buf[:, :cols] = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return buf[:, :cols]


def stored(m, n, k, ta, tb, gen, seed):
    A = gen(k, m, seed) if ta else gen(m, k, seed)
    B = gen(n, k, seed + 1) if tb else gen(k, n, seed + 1)
    return A, B


def run(A, B, C, alpha, beta, ta, tb, levels, variant, dtype="f64"):
    dC = dev(C)
    sg.dgemm(dev(A), dev(B), dC, alpha=alpha, beta=beta, trans_a=ta, trans_b=tb, levels=levels,
             variant=variant, dtype=dtype)
    torch.cuda.synchronize()
    assert sg.strassen_device_status(0) == 0
    return dC.cpu().numpy()


@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("levels,variant", [(0, "ABC"), (1, "ABC"), (1, "AB"), (1, "NAIVE"), (2, "ABC"),
                                            (2, "AB"), (2, "NAIVE"), (3, "ABC"), (2, "HYBRID"), (3, "HYBRID")])
def test_integer_bit_exact(ta, tb, levels, variant):
    m, n, k = 301, 263, 418
    A, B = stored(m, n, k, ta, tb, W.integer, 10)
    C = W.integer(m, n, 12)
    ref = oracle.dgemm(ta, tb, 3.0, A, B, -2.0, C)
    got = run(A, B, C, 3.0, -2.0, ta, tb, levels, variant)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("ta,tb", [(1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("levels", [0, 2])
def test_float_tolerance(ta, tb, levels):
    m, n, k = 384, 320, 512
    A, B = stored(m, n, k, ta, tb, W.uniform, 20)
    C = W.uniform(m, n, 22)
    alpha, beta = 0.75, -1.25
    ref = oracle.dgemm(ta, tb, alpha, A, B, beta, C)
    got = run(A, B, C, alpha, beta, ta, tb, levels, "ABC")
    Aop = A.T if ta else A
    Bop = B.T if tb else B
    den = abs(alpha) * float(np.max(np.sum(np.abs(Aop), axis=1))) * float(np.max(np.abs(Bop)))
    assert float(np.max(np.abs(got - ref))) / den <= TOL[levels]


def test_beta_zero_ignores_nan_and_alpha_zero_only_scales():
    m, n, k = 130, 90, 70
    A, B = stored(m, n, k, 1, 0, W.integer, 30)
    Cnan = np.full((m, n), np.nan)
    got = run(A, B, Cnan, 2.0, 0.0, 1, 0, 2, "ABC")
    assert np.array_equal(got, 2.0 * (A.T @ B))
    C = W.integer(m, n, 32)
    assert np.array_equal(run(A, B, C, 0.0, 3.0, 1, 0, 1, "ABC"), 3.0 * C)


def test_transposed_operands_with_padded_leading_dimensions():
    m, n, k = 97, 131, 77
    A, B = stored(m, n, k, 1, 1, W.integer, 40)
    C = W.integer(m, n, 42)
    ref = oracle.dgemm(1, 1, 1.0, A, B, 1.0, C)
    for levels in (0, 1, 2):
        dA, dB = dev(A, ld=m + 3), dev(B, ld=k + 5)
        cbuf = torch.full((m, n + 7), 777.0, dtype=torch.float64, device="cuda")
        cbuf[:, :n] = torch.from_numpy(C).cuda()
        sg.dgemm(dA, dB, cbuf[:, :n], trans_a=True, trans_b=True, levels=levels)
        torch.cuda.synchronize()
        got = cbuf.cpu().numpy()
        assert np.array_equal(got[:, :n], ref), levels
        assert np.all(got[:, n:] == 777.0)


@pytest.mark.parametrize("ta,tb", [(1, 0), (0, 1)])
def test_split_precision_with_transposes(ta, tb):
    """The split works on op(A) and op(B); alpha = 2 scales every partial product by a
    power of two, which the scheme carries exactly (as doubling op(A))."""
    m, n, k = 150, 140, 260
    A, B = stored(m, n, k, ta, tb, W.uniform, 50)
    C = W.uniform(m, n, 52)
    Aop = np.ascontiguousarray(A.T if ta else A)
    Bop = np.ascontiguousarray(B.T if tb else B)
    for levels in (0, 1):
        assert np.array_equal(run(A, B, C, 1.0, 1.0, ta, tb, levels, "ABC", "oz_bf16"),
                              ozaki.gemm(Aop, Bop, C, levels))
        assert np.array_equal(run(A, B, C, 2.0, 1.0, ta, tb, levels, "ABC", "oz_bf16"),
                              ozaki.gemm(2.0 * Aop, Bop, C, levels))


def test_argument_checks():
    P = 0x1000
    # lda must cover the stored rows of A^T (m = 8 columns)
    assert sg.strassen_dgemm(1, 0, 8, 4, 4, 1.0, P, 4, 2 * P, 4, 1.0, 3 * P, 4, 1, 0, 0, 0) == -2
    assert sg.strassen_dgemm(2, 0, 8, 4, 4, 1.0, P, 8, 2 * P, 4, 1.0, 3 * P, 4, 1, 0, 0, 0) == -9
    assert sg.strassen_dgemm(0, 0, 0, 4, 4, 1.0, 0, 4, 0, 4, 1.0, 0, 4, 1, 0, 0, 0) == 0
