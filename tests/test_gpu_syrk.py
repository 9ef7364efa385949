"""strassen_dsyrk (symmetric rank-k update on one triangle, Strassen on the off-diagonal
blocks) against the oracle's definition, through the C ABI.

* Integer-valued inputs: every sum and product is exact, so the triangle must equal the
  oracle bit for bit, for both triangles, both transposes, several Strassen levels and
  shapes that exercise the recursion (n above 1024) and ragged splits.
* The other triangle holds NaN and must come back untouched.
* Uniform[-1, 1] inputs: the strict max-norm error against the exact product stays
  within the two-level bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1605_01078_gb300 as sg
import workloads as W

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def tri_mask(n, uplo):
    i, j = np.indices((n, n))
    return (j <= i) if uplo == 0 else (j >= i)


@pytest.mark.parametrize("n,k", [(1, 1), (13, 7), (300, 129), (1030, 200), (2500, 96)])
@pytest.mark.parametrize("uplo", [0, 1])
@pytest.mark.parametrize("trans", [0, 1])
@pytest.mark.parametrize("levels", [0, 2, -1])
def test_dsyrk_integer_bit_exact(n, k, uplo, trans, levels):
    A = W.integer(k, n, 1) if trans else W.integer(n, k, 1)
    C = W.integer(n, n, 2)
    mask = tri_mask(n, uplo)
    C[~mask] = np.nan
    ref = oracle.dsyrk(uplo, trans, 2.0, A, -1.0, C)
    dC = dev(C)
    sg.dsyrk(dev(A), dC, alpha=2.0, beta=-1.0, lower=(uplo == 0), trans=bool(trans), levels=levels)
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    assert np.array_equal(got[mask], ref[mask])
    assert np.all(np.isnan(got[~mask]))


def test_dsyrk_beta_zero_alpha_zero_and_empty():
    n, k = 40, 9
    A = W.integer(n, k, 3)
    C = np.full((n, n), np.nan)
    dC = dev(C)
    sg.dsyrk(dev(A), dC, alpha=1.0, beta=0.0, lower=True)
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    mask = tri_mask(n, 0)
    assert np.array_equal(got[mask], (A @ A.T)[mask]) and np.all(np.isnan(got[~mask]))
    C2 = W.integer(n, n, 4)
    dC2 = dev(C2)
    sg.dsyrk(dev(A), dC2, alpha=0.0, beta=3.0, lower=False)
    torch.cuda.synchronize()
    up = tri_mask(n, 1)
    assert np.array_equal(dC2.cpu().numpy()[up], 3.0 * C2[up])
    assert np.array_equal(dC2.cpu().numpy()[~up], C2[~up])
    assert sg.strassen_dsyrk(0, 0, 0, 4, 1.0, 0, 4, 1.0, 0, 1, -1, 0, 0) == 0


@pytest.mark.parametrize("uplo", [0, 1])
def test_dsyrk_float_strict_error_and_determinism(uplo):
    n, k = 3000, 2048
    A = W.uniform(n, k, 5)
    C = W.uniform(n, n, 6)
    mask = tri_mask(n, uplo)
    rows, cols = np.nonzero(mask)
    g = np.random.Generator(np.random.Philox(7))
    pick = g.choice(rows.size, 2048, replace=False)
    rows, cols = rows[pick], cols[pick]
    exact = oracle.gemm_sampled(A, np.ascontiguousarray(A.T), C, rows, cols)
    outs = []
    for _ in range(2):
        dC = dev(C)
        sg.dsyrk(dev(A), dC, lower=(uplo == 0), levels=2, deterministic=True)
        torch.cuda.synchronize()
        outs.append(dC.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    err = float(np.max(np.abs(outs[0][rows, cols] - exact))) / (float(np.max(np.abs(A))) ** 2)
    assert err <= 1e-12
    assert np.array_equal(outs[0][~mask], C[~mask])
