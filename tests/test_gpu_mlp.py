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
                     g.integers(0, 3, n), base=g.normal(-6, 3, size=(n, ref.N_OUT)))
    T = g.normal(0, 0.5, size=(n, ref.N_OUT))
    M = (g.uniform(size=(n, ref.N_OUT)) < 0.7).astype(np.float64)
    M[0, 0] = 1.0
    theta = ref.init(seed) + g.normal(0, 0.05, ref.N_PARAMS)
    return X, T, M, theta


def d32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_param_count():
    assert sg.strassen_mlp_param_count() == ref.N_PARAMS


def test_forward_matches_oracle():
    X, _, _, theta = batch(1)
    Y = torch.empty((X.shape[0], ref.N_OUT), dtype=torch.float32, device="cuda")
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


def test_features_follow_the_definition():
    """The library's selector features are the oracle's definition applied to the
    library's model values; the model is the library's strassen_model_seconds for the
    candidate's level and variant (its best tile)."""
    for (m, n, k, d) in ((4096, 4096, 4096, 0), (300, 5000, 777, 0), (8192, 1024, 2048, 2)):
        x, base, valid = sg.strassen_selector_features(m, n, k, d)
        want = ref.features([m], [n], [k], [d], base=[base])[0]
        assert np.allclose(np.array(x), want, atol=1e-6)
        cands = tune.candidates()
        assert valid == sum(1 << c for c in tune.valid_candidates(d))
        if d == 0:  # the two tiles of a (levels, variant): their minimum is the model's figure
            for c in range(0, len(cands), 2):
                lv, var, tile = cands[c]
                assert cands[c + 1] == (lv, var, 1) and tile == 0
                best = min(2.0 ** base[c], 2.0 ** base[c + 1])
                assert best == pytest.approx(sg.strassen_model_seconds(m, n, k, lv, var), rel=1e-5)


def test_training_reduces_loss_on_a_teacher_network():
    g = np.random.Generator(np.random.Philox(4))
    rows = []
    teacher = ref.init(99)
    teacher[-(ref.N_OUT * (ref.N_H + 1)):] = g.normal(0, 0.1, ref.N_OUT * (ref.N_H + 1))
    for _ in range(200):
        m, n, k = (int(v) for v in g.integers(256, 16384, 3))
        d = int(g.choice([0, 2]))
        x, base, valid = sg.strassen_selector_features(m, n, k, d)
        y, _ = ref.forward(teacher, np.array([x], dtype=np.float64))
        times = [float(2.0 ** (base[c] + y[0, c])) if (valid >> c) & 1 else float("nan")
                 for c in range(ref.N_OUT)]
        rows.append({"m": m, "n": n, "k": k, "dtype": d, "times": times})
    params, hist = tune.train(rows, steps=800, lr=3e-3, seed=0)
    assert hist[-1][1] < 0.1 * hist[0][1]


def test_select_uses_the_loaded_network():
    """With zero weights the network's output is b3: a large negative correction for one
    candidate makes it the choice (among the dtype's valid candidates)."""
    sg.strassen_tune_clear()
    p = np.zeros(ref.N_PARAMS, dtype=np.float32)
    b3 = ref.N_PARAMS - ref.N_OUT
    p[b3 + 7] = -100.0    # (1 level, Naive, 64-wide tile): FP64 only
    p[b3 + 8] = -50.0     # (2 levels, ABC, 128-wide tile): valid for split precision too
    arr = np.ascontiguousarray(p)
    assert sg.strassen_selector_load(arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), arr.size) == 0
    try:
        assert sg.strassen_select(4096, 4096, 4096, sg.STRASSEN_F64) == (1, sg.STRASSEN_NAIVE, 1)
        assert sg.strassen_select(4096, 4096, 4096, sg.STRASSEN_F64_OZ_BF16) == (2, sg.STRASSEN_ABC, 0)
        # an exhaustive record takes precedence
        assert sg.strassen_tune_record(4096, 4096, 4096, 0, 0, 0, 0) == 0
        assert sg.strassen_select(4096, 4096, 4096, sg.STRASSEN_F64) == (0, sg.STRASSEN_ABC, 0)
        # the network disabled for a dtype: the analytic model answers
        sg.strassen_tune_clear()
        assert sg.strassen_selector_use(sg.STRASSEN_F64, 0) == 0
        assert sg.strassen_select(4096, 4096, 4096, sg.STRASSEN_F64) != (1, sg.STRASSEN_NAIVE, 1)
    finally:
        sg.strassen_tune_clear()
        sg.strassen_selector_clear()
    lv, var, _ = sg.strassen_select(8192, 8192, 8192, sg.STRASSEN_F64)
    assert lv == 3  # back to the analytic model (three levels at 8192^3)


def test_auto_call_under_capture_uses_cached_choice_only():
    """Inside a stream capture, an automatic call takes the network's choice only from
    its cache (no launch, no wait): the captured graph then runs that plan."""
    p = np.zeros(ref.N_PARAMS, dtype=np.float32)
    p[ref.N_PARAMS - ref.N_OUT + 2] = -100.0  # (1 level, ABC, 128-wide tile)
    arr = np.ascontiguousarray(p)
    assert sg.strassen_selector_load(arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), arr.size) == 0
    try:
        A = torch.ones((512, 512), dtype=torch.float64, device="cuda")
        B = torch.ones((512, 512), dtype=torch.float64, device="cuda")
        C = torch.zeros((512, 512), dtype=torch.float64, device="cuda")
        assert sg.strassen_select(512, 512, 512, sg.STRASSEN_F64) == (1, sg.STRASSEN_ABC, 0)  # cached now
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            sg.gemm(A, B, C, levels=-1, variant="AUTO")
        C.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.all(C == 512.0)
    finally:
        sg.strassen_selector_clear()
