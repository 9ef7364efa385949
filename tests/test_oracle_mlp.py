"""Pins of the selector-MLP oracle: gradients against central finite differences, the
forward pass against a hand-computed tiny network, the masked loss, and Adam against
its closed-form first step (no GPU)."""
import numpy as np

from oracle import mlp


def data(seed, batch=9):
    g = np.random.Generator(np.random.Philox(seed))
    X = mlp.features(g.integers(256, 16384, batch), g.integers(256, 16384, batch), g.integers(256, 16384, batch),
                     g.integers(0, 3, batch))
    T = g.normal(-5, 2, size=(batch, mlp.N_OUT))
    mask = (g.uniform(size=(batch, mlp.N_OUT)) < 0.7).astype(np.float64)
    mask[0, 0] = 1.0
    return X, T, mask


def test_gradient_matches_finite_differences():
    X, T, mask = data(1)
    theta = mlp.init(3) + np.random.Generator(np.random.Philox(4)).normal(0, 0.05, mlp.N_PARAMS)
    g = mlp.grad(theta, X, T, mask)
    rng = np.random.Generator(np.random.Philox(5))
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    for i in idx:
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, X, T, mask) - mlp.loss(tm, X, T, mask)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_forward_of_a_hand_built_network():
    theta = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(theta)  # views are copies; build by offsets instead
    # W1[0,0] = 1, b1[1] = -1; W2[0,0] = 2; W3[c,0] = c; b3 = 0.5
    o = 0
    sizes = {n: int(np.prod(s)) for n, s in mlp.SHAPES}
    offs = {}
    for n, _ in mlp.SHAPES:
        offs[n] = o
        o += sizes[n]
    theta[offs["W1"] + 0] = 1.0
    theta[offs["b1"] + 1] = -1.0
    theta[offs["W2"] + 0] = 2.0
    for c in range(mlp.N_OUT):
        theta[offs["W3"] + c * mlp.N_H] = float(c)
        theta[offs["b3"] + c] = 0.5
    X = np.zeros((2, mlp.N_IN))
    X[0, :6] = [1.5, 0, 0, 1, 0, 0]
    X[1, :6] = [-1.0, 0, 0, 0, 1, 0]
    y, _ = mlp.forward(theta, X)
    # h1[0] = relu(x0) ; h2[0] = relu(2 h1[0]) ; y_c = c * h2[0] + 0.5
    assert np.allclose(y[0], np.arange(mlp.N_OUT) * 3.0 + 0.5)
    assert np.allclose(y[1], np.full(mlp.N_OUT, 0.5))
    assert p["W1"].shape == (64, 22) and p["W3"].shape == (16, 64)


def test_masked_loss_ignores_unmeasured_candidates():
    X, T, mask = data(2)
    theta = mlp.init(1)
    y, _ = mlp.forward(theta, X)
    T2 = T.copy()
    T2[mask == 0] = 1e6
    assert mlp.loss(theta, X, T, mask) == mlp.loss(theta, X, T2, mask)
    assert np.isclose(mlp.loss(theta, X, y, mask), 0.0)


def test_adam_first_step_is_lr_times_sign():
    theta = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    new, m, v = mlp.adam(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.1)
    # bias-corrected m/sqrt(v) = g/|g| on the first step (up to eps)
    assert np.allclose(new, theta - 0.1 * np.sign(g), atol=1e-6)


def test_features():
    x = mlp.features([2048], [256], [16384], [2])
    assert np.allclose(x[0, :6], [0.0, -1.0, 1.0, 0, 0, 1]) and np.allclose(x[0, 6:], 1.0)
    b = np.arange(16, dtype=np.float64) - 10.0
    x = mlp.features([4096], [4096], [4096], [0], base=[b])
    assert np.allclose(x[0, 6:], (b + 7.0) / 7.0) and x.shape == (1, 22)
