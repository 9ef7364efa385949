"""The learned selector: training with the library's kernels on live timings, and the
shipped network's gain over the selection without it on the committed held-out timings.

The selection without the network is the analytic model (FP64) or classical slices
(split precision).  The network predicts a correction to the model's log2 seconds for
each of the 16 candidates (levels 0-2 of ABC/AB/Naive and three-level ABC, each with the
128- or 64-wide tile).
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1605_01078_gb300 as sg
from paper_1605_01078_gb300 import tune
import workloads as W

pytestmark = pytest.mark.gpu

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1605_01078_gb300", "data")


def test_training_on_live_timings():
    """Exhaustive timing of 32 small seeded shapes (all 16 candidates), full-batch Adam
    with the library's kernels: the loss falls, and once loaded, strassen_select returns
    the network's argmin."""
    shapes = W.loguniform_shapes(32, seed=11, lo=128, hi=2048)
    timer = tune.Timer(2048 * 2048, 2048 * 2048, 2048 * 2048)
    rows = tune.measure(shapes, sg.STRASSEN_F64, timer)
    assert all(np.isfinite(r["times"]).all() for r in rows)
    params, hist = tune.train(rows, steps=1500, lr=1e-3, seed=0)
    assert hist[-1][1] < hist[0][1]
    choices = tune.choose_mlp(params, rows)
    r_mlp = tune.regret(rows, choices)
    r_fixed = tune.regret(rows, tune.choose_fixed(rows, 2))
    print("training shapes: regret mlp", r_mlp, "always 1L ABC", r_fixed)
    assert r_mlp["mean"] <= r_fixed["mean"]
    cl = tune.candidates()
    tune.load_selector(params)
    try:
        for r, c in zip(rows[:8], choices[:8]):
            assert sg.strassen_select(r["m"], r["n"], r["k"], sg.STRASSEN_F64) == cl[c]
    finally:
        sg.strassen_selector_clear()


def test_shipped_network_gain_on_heldout_shapes():
    """The shipped network against the selection without it on the committed held-out
    timings (1000 FP64 and 200 split-precision shapes, m, n, k log-uniform in [256,
    16384], seeds 2 and 4, every candidate timed): it ships enabled for a dtype exactly
    when its mean regret there is below the method without it, and the shipped
    metadata's figures are what these rows give."""
    meta = json.load(open(os.path.join(DATA, "selector_gb300.json")))
    rows = json.load(open(os.path.join(DATA, "selector_gb300_heldout_rows.json")))
    params = np.array(meta["params"], dtype=np.float32)
    assert params.size == sg.strassen_mlp_param_count()
    for d, name in ((sg.STRASSEN_F64, "f64"), (sg.STRASSEN_F64_OZ_BF16, "oz_bf16")):
        sub = [r for r in rows if r["dtype"] == d]
        r_mlp = tune.regret(sub, tune.choose_mlp(params, sub))
        r_without = tune.regret(sub, tune.choose_model(sub))
        print(name, len(sub), "shapes: regret mlp", r_mlp, "without the network", r_without)
        assert len(sub) >= (1000 if d == sg.STRASSEN_F64 else 200)
        assert meta["use_for_dtype"][str(d)] == (r_mlp["mean"] < r_without["mean"])
        assert r_mlp["mean"] == pytest.approx(meta["heldout_regret_mean"][name]["mlp"], abs=2e-4)


def test_shipped_selector_loads():
    meta = tune.load_default_selector()
    try:
        for d in (sg.STRASSEN_F64, sg.STRASSEN_F64_OZ_BF16):
            lv, var, tile = sg.strassen_select(8192, 8192, 8192, d)
            assert (lv, var, tile) in [tune.candidates()[c] for c in tune.valid_candidates(d)]
        assert isinstance(meta["use_for_dtype"]["0"], bool)
    finally:
        sg.strassen_selector_clear()
