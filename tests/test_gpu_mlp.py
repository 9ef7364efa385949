"""The selector MLP's CUDA kernels (forward, loss gradient, Adam, selection) against
the FP64 oracle of the same network, through the C ABI."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as ref
import paper_1605_01078_gb300 as sg
from paper_1605_01078_gb300 import tune

pytestmark = pytest.mark.gpu


def batch(seed, n=37):
    g = np.random.Generator(np.random.Philox(seed))
    X = ref.features(g.integers(256, 16384, n), g.integers(256, 16384, n), g.integers(256, 16384, n),
                     g.integers(0, 3, n))
    T = g.normal(-5, 2, size=(n, 7))
    M = (g.uniform(size=(n, 7)) < 0.7).astype(np.float64)
    M[0, 0] = 1.0
    theta = ref.init(seed) + g.normal(0, 0.05, ref.N_PARAMS)
    return X, T, M, theta


def d32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_param_count():
    assert sg.strassen_mlp_param_count() == ref.N_PARAMS


def test_forward_matches_oracle():
    X, _, _, theta = batch(1)
    Y = torch.empty((X.shape[0], 7), dtype=torch.float32, device="cuda")
    dP, dX = d32(theta), d32(X)  # keep the device copies alive until the kernel has run
    assert sg.strassen_mlp_forward(dP.data_ptr(), dX.data_ptr(), X.shape[0], Y.data_ptr(), 0) == 0
    torch.cuda.synchronize()
    want, _ = ref.forward(theta.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(Y.cpu().numpy() - want)) <= 1e-4 * max(1.0, np.max(np.abs(want)))


def test_gradient_matches_oracle():
    X, T, M, theta = batch(2)
    G = torch.empty(ref.N_PARAMS, dtype=torch.float32, device="cuda")
    dP, dX, dT, dM = d32(theta), d32(X), d32(T), d32(M)
    st = sg.strassen_mlp_loss_grad(dP.data_ptr(), dX.data_ptr(), dT.data_ptr(), dM.data_ptr(),
                                   X.shape[0], float(M.sum()), G.data_ptr(), 0)
    assert st == 0
    torch.cuda.synchronize()
    th32 = theta.astype(np.float32).astype(np.float64)
    want = ref.grad(th32, X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64), M)
    got = G.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - want)) <= 2e-4 * max(1.0, np.max(np.abs(want)))


def test_adam_matches_oracle():
    g = np.random.Generator(np.random.Philox(3))
    n = 1000
    p, m, v = g.normal(size=n), np.zeros(n), np.zeros(n)
    P, Mo, V = d32(p), d32(m), d32(v)
    for step in (1, 2, 3):
        grad = g.normal(size=n)
        dG = d32(grad)
        assert sg.strassen_mlp_adam(P.data_ptr(), dG.data_ptr(), Mo.data_ptr(), V.data_ptr(), n, step,
                                    0.01, 0) == 0
        torch.cuda.synchronize()
        p, m, v = ref.adam(p, grad, m, v, step, lr=0.01)
    torch.cuda.synchronize()
    assert np.max(np.abs(P.cpu().numpy() - p)) <= 1e-5


def test_training_reduces_loss_on_a_teacher_network():
    g = np.random.Generator(np.random.Philox(4))
    rows = []
    teacher = ref.init(99)
    for _ in range(200):
        m, n, k = (int(v) for v in g.integers(256, 16384, 3))
        d = int(g.choice([0, 2]))
        y, _ = ref.forward(teacher, ref.features([m], [n], [k], [d]))
        times = [float(2.0 ** y[0, c]) if c in tune.VALID[d] else float("nan") for c in range(7)]
        rows.append({"m": m, "n": n, "k": k, "dtype": d, "times": times})
    params, hist = tune.train(rows, steps=800, lr=3e-3, seed=0)
    assert hist[-1][1] < 0.1 * hist[0][1]


def test_select_uses_the_loaded_network():
    sg.strassen_tune_clear()
    p = np.zeros(ref.N_PARAMS, dtype=np.float32)
    b3 = ref.N_PARAMS - 7
    p[b3:] = [3, 3, 3, -3, -1, 3, 3]
    arr = np.ascontiguousarray(p)
    assert sg.strassen_selector_load(arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), arr.size) == 0
    try:
        assert sg.strassen_select(4096, 4096, 4096, sg.STRASSEN_F64) == (1, sg.STRASSEN_NAIVE, 0)
        # split precision: only levels 0, 1, 2 of ABC are candidates
        assert sg.strassen_select(4096, 4096, 4096, sg.STRASSEN_F64_OZ_BF16) == (2, sg.STRASSEN_ABC, 0)
        # an exhaustive record takes precedence
        assert sg.strassen_tune_record(4096, 4096, 4096, 0, 0, 0, 0) == 0
        assert sg.strassen_select(4096, 4096, 4096, sg.STRASSEN_F64) == (0, sg.STRASSEN_ABC, 0)
    finally:
        sg.strassen_tune_clear()
        sg.strassen_selector_clear()
    lv, var, _ = sg.strassen_select(8192, 8192, 8192, sg.STRASSEN_F64)
    assert lv == 3  # back to the analytic model (three levels at 8192^3)
