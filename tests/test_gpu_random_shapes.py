"""Randomised parity sweep (seeded): shapes from 1 to 700 along each dimension with
extreme aspect ratios, every level 0-3 and variant, transposes, integer alpha and beta,
padded leading dimensions, both block tiles (via the launch's own choice) -- integer
inputs, so every result must equal the oracle's definition bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1605_01078_gb300 as sg
import workloads as W

pytestmark = pytest.mark.gpu

VARIANTS = ["ABC", "AB", "NAIVE"]


def cases(count=48, seed=2024):
    g = np.random.Generator(np.random.Philox(seed))
    out = []
    for i in range(count):
        kind = i % 4
        if kind == 0:      # small and ragged
            m, n, k = (int(x) for x in g.integers(1, 80, size=3))
        elif kind == 1:    # tall or wide
            m, n, k = int(g.integers(1, 12)), int(g.integers(200, 700)), int(g.integers(1, 400))
            if g.integers(0, 2):
                m, n = n, m
        elif kind == 2:    # long reduction
            m, n, k = int(g.integers(1, 60)), int(g.integers(1, 60)), int(g.integers(300, 700))
        else:              # mid-size
            m, n, k = (int(x) for x in g.integers(100, 500, size=3))
        levels = int(g.integers(0, 4))
        variant = VARIANTS[int(g.integers(0, 3))]
        ta, tb = int(g.integers(0, 2)), int(g.integers(0, 2))
        alpha = float(g.integers(-3, 4))
        beta = float(g.integers(-2, 3))
        pad_a, pad_b, pad_c = (int(x) for x in g.integers(0, 5, size=3))
        out.append((m, n, k, levels, variant, ta, tb, alpha, beta, pad_a, pad_b, pad_c))
    return out


def dev(x, pad):
    rows, cols = x.shape
    buf = torch.full((rows, cols + pad), float("nan"), dtype=torch.float64, device="cuda")
    buf[:, :cols] = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return buf[:, :cols]


@pytest.mark.parametrize("case", cases(), ids=lambda c: "x".join(str(v) for v in c[:3]) + f"-L{c[3]}{c[4]}")
def test_random_shape_bit_exact(case):
    m, n, k, levels, variant, ta, tb, alpha, beta, pad_a, pad_b, pad_c = case
    A = W.integer(k, m, 1) if ta else W.integer(m, k, 1)
    B = W.integer(n, k, 2) if tb else W.integer(k, n, 2)
    C = W.integer(m, n, 3)
    ref = oracle.dgemm(ta, tb, alpha, A, B, beta, C)
    dC = dev(C, pad_c)
    sg.dgemm(dev(A, pad_a), dev(B, pad_b), dC, alpha=alpha, beta=beta, trans_a=bool(ta), trans_b=bool(tb),
             levels=levels, variant=variant)
    torch.cuda.synchronize()
    assert sg.strassen_device_status(0) == 0
    assert np.array_equal(dC.cpu().numpy(), ref)
