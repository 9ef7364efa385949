"""Exhaustive autotuner and learned-selector training for the Strassen library.

The family of Section 4.1 has one member per (levels, variant); which one is fastest
depends on the shape (the paper draws this conclusion from its model and its
measurements).  This module

* times the candidates of a shape through the C ABI (``measure``) -- the exhaustive
  search, whose winners ``record`` hands to the library (strassen_tune_record);
* trains the selector MLP on such timings with the library's own CUDA kernels
  (strassen_mlp_loss_grad / strassen_mlp_adam), loads it (strassen_selector_load), and
* evaluates choices by regret t(chosen) / t(best) - 1 against exhaustive timing, for
  the MLP, the analytic model (strassen_model_seconds) and fixed rules.

Python only drives the calls; all arithmetic of the network runs in the CUDA kernels.
"""
from __future__ import annotations

import ctypes
import json
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import _binding as B

NC = B.SELECTOR_CANDIDATES  # the network's outputs: candidate c -> (levels, variant, tile)


def candidates() -> List[Tuple[int, int, int]]:
    return [B.strassen_selector_candidate(c) for c in range(NC)]


def valid_candidates(dtype: int) -> List[int]:
    _, _, mask = B.strassen_selector_features(1024, 1024, 1024, dtype)
    return [c for c in range(NC) if (mask >> c) & 1]


DTYPE_NAME = {B.STRASSEN_F64: "f64", B.STRASSEN_F64_OZ_BF16: "oz_bf16"}


def features(rows) -> Tuple[np.ndarray, np.ndarray]:
    """Network inputs X [rows, 22] and the analytic model's log2 seconds [rows, 16], as
    the library computes them (strassen_selector_features)."""
    X = np.zeros((len(rows), B.SELECTOR_INPUTS), dtype=np.float32)
    base = np.zeros((len(rows), NC), dtype=np.float32)
    for i, r in enumerate(rows):
        x, b, _ = B.strassen_selector_features(r["m"], r["n"], r["k"], r["dtype"])
        X[i], base[i] = x, b
    return X, base


class Timer:
    """Times candidates on one preallocated set of operand buffers."""

    def __init__(self, max_elems_a: int, max_elems_b: int, max_elems_c: int):
        import torch
        self.torch = torch
        self.A = torch.rand(max_elems_a, dtype=torch.float64, device="cuda") * 2 - 1
        self.B = torch.rand(max_elems_b, dtype=torch.float64, device="cuda") * 2 - 1
        self.C = torch.zeros(max_elems_c, dtype=torch.float64, device="cuda")
        self.stream = torch.cuda.current_stream()
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)

    def _call(self, m, n, k, dtype):
        st = B.strassen_gemm(m, n, k, self.A.data_ptr(), k, self.B.data_ptr(), n, self.C.data_ptr(), n,
                             -1, B.STRASSEN_AUTO, dtype, self.stream.cuda_stream)
        if st != 0:
            raise B.StrassenError(st, "strassen_gemm")

    def time(self, m, n, k, levels, variant, tile, dtype, min_seconds=2e-3, max_reps=20,
             single_above=0.02) -> float:
        """Seconds per call of exactly (levels, variant, tile) -- fixed by an exhaustive
        record for the shape, which the automatic call follows.  A first call of at least
        `single_above` seconds is the measurement; shorter ones are repeated (the first
        discarded) until `min_seconds` of work or `max_reps` calls."""
        st = B.strassen_tune_record(m, n, k, dtype, levels, variant, tile)
        if st != 0:
            raise B.StrassenError(st, "strassen_tune_record")
        try:
            self.e0.record(self.stream)
            self._call(m, n, k, dtype)
            self.e1.record(self.stream)
            self.e1.synchronize()
            first = self.e0.elapsed_time(self.e1) / 1e3
            if first >= single_above:
                return first
            reps, total = 0, 0.0
            while reps < max_reps and (total < min_seconds or reps == 0):
                self.e0.record(self.stream)
                self._call(m, n, k, dtype)
                self.e1.record(self.stream)
                self.e1.synchronize()
                total += self.e0.elapsed_time(self.e1) / 1e3
                reps += 1
            return total / reps
        finally:
            B.strassen_tune_clear()


def measure(shapes: Sequence[Tuple[int, int, int]], dtype: int, timer: Timer,
            cands: Optional[Sequence[int]] = None, log_path: Optional[str] = None) -> List[Dict]:
    """Exhaustive timing: one row per shape with the seconds of every valid candidate
    (NaN for the others).  Candidates whose levels would be clamped for the shape are
    timed as what they run.  With log_path, every row is also appended to that file as
    one JSON line as soon as it is measured."""
    cl = candidates()
    cs = list(valid_candidates(dtype) if cands is None else cands)
    rows = []
    for (m, n, k) in shapes:
        times = [math.nan] * NC
        for c in cs:
            lv, var, tile = cl[c]
            times[c] = timer.time(m, n, k, lv, var, tile, dtype)
        row = {"m": int(m), "n": int(n), "k": int(k), "dtype": int(dtype), "times": times}
        rows.append(row)
        if log_path:
            with open(log_path, "a") as fh:
                fh.write(json.dumps(row) + "\n")
    return rows


def best_of(row) -> int:
    t = np.array(row["times"], dtype=np.float64)
    return int(np.nanargmin(t))


def record(rows) -> None:
    """Hand the exhaustive winners to the library's selection table."""
    cl = candidates()
    for r in rows:
        lv, var, tile = cl[best_of(r)]
        st = B.strassen_tune_record(r["m"], r["n"], r["k"], r["dtype"], lv, var, tile)
        if st != 0:
            raise B.StrassenError(st, "strassen_tune_record")


def arrays(rows):
    """Network inputs X, targets T = log2 measured seconds - the model's log2 seconds
    (the correction the network learns), the mask of measured candidates, and the
    model's log2 seconds."""
    X, base = features(rows)
    t = np.array([r["times"] + [math.nan] * (NC - len(r["times"])) for r in rows], dtype=np.float64)
    ok = np.isfinite(t)
    mask = ok.astype(np.float32)
    T = np.where(ok, np.log2(np.where(ok, t, 1.0)) - base, 0.0).astype(np.float32)
    return X, T, mask, base


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights for the hidden layers, zero output layer (float32), in the
    library's parameter order: the untrained network predicts no correction, i.e. it
    starts as the analytic model."""
    g = np.random.Generator(np.random.Philox(seed))
    shapes = [(64, B.SELECTOR_INPUTS), (64,), (64, 64), (64,), (NC, 64), (NC,)]
    parts = []
    for i, shp in enumerate(shapes):
        if len(shp) == 2 and i < 4:
            lim = math.sqrt(6.0 / shp[1])
            parts.append(g.uniform(-lim, lim, size=shp).ravel())
        else:
            parts.append(np.zeros(shp).ravel())
    return np.concatenate(parts).astype(np.float32)


def train(rows, steps: int = 3000, lr: float = 3e-3, seed: int = 0, params: Optional[np.ndarray] = None):
    """Full-batch Adam on the masked MSE of log2 times, entirely in the library's
    kernels.  Returns (parameters as numpy float32, loss history: step 0, then every
    100 steps)."""
    import torch
    X, T, mask, _ = arrays(rows)
    n_par = B.strassen_mlp_param_count()
    p0 = init_params(seed) if params is None else np.asarray(params, dtype=np.float32)
    assert p0.size == n_par
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dX, dT, dM = dev(X), dev(T), dev(mask)
    P = dev(p0)
    G = torch.zeros_like(P)
    Mo = torch.zeros_like(P)
    V = torch.zeros_like(P)
    Y = torch.empty((len(rows), NC), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    msum = float(mask.sum())
    hist = []

    def current_loss():
        B.strassen_mlp_forward(P.data_ptr(), dX.data_ptr(), len(rows), Y.data_ptr(), s)
        return float(((Y - dT) ** 2 * dM).sum() / msum)

    hist.append((0, current_loss()))
    for step in range(1, steps + 1):
        st = B.strassen_mlp_loss_grad(P.data_ptr(), dX.data_ptr(), dT.data_ptr(), dM.data_ptr(), len(rows), msum,
                                      G.data_ptr(), s)
        if st != 0:
            raise B.StrassenError(st, "strassen_mlp_loss_grad")
        st = B.strassen_mlp_adam(P.data_ptr(), G.data_ptr(), Mo.data_ptr(), V.data_ptr(), n_par, step, lr, s)
        if st != 0:
            raise B.StrassenError(st, "strassen_mlp_adam")
        if step % 100 == 0 or step == steps:
            hist.append((step, current_loss()))
    return P.cpu().numpy(), hist


def predict(params: np.ndarray, rows) -> np.ndarray:
    """Predicted log2 seconds [rows, 20]: the model's plus the network's correction (the
    library's forward kernel)."""
    import torch
    X, _, _, base = arrays(rows)
    P = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).cuda()
    dX = torch.from_numpy(X).cuda()
    Y = torch.empty((len(rows), NC), dtype=torch.float32, device="cuda")
    st = B.strassen_mlp_forward(P.data_ptr(), dX.data_ptr(), len(rows), Y.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    if st != 0:
        raise B.StrassenError(st, "strassen_mlp_forward")
    return Y.cpu().numpy() + base


def choose_mlp(params, rows) -> List[int]:
    Y = predict(params, rows)
    out = []
    for r, y in zip(rows, Y):
        valid = valid_candidates(r["dtype"])
        out.append(int(valid[int(np.argmin(y[valid]))]))
    return out


def choose_model(rows) -> List[int]:
    """The selection without the network: the analytic model's choice for FP64 (its own
    argmin with the 1 % tie-break, as strassen_select returns it), classical slices for
    split precision."""
    cl = candidates()
    out = []
    B.strassen_selector_use(B.STRASSEN_F64, 0)  # a loaded network must not answer here
    try:
        for r in rows:
            if r["dtype"] != B.STRASSEN_F64:
                out.append(0)
                continue
            out.append(cl.index(B.strassen_select(r["m"], r["n"], r["k"], r["dtype"])))
    finally:
        B.strassen_selector_use(B.STRASSEN_F64, 1)
    return out


def choose_fixed(rows, candidate: int) -> List[int]:
    return [candidate if candidate in valid_candidates(r["dtype"]) else 0 for r in rows]


def regret(rows, choices) -> Dict[str, float]:
    """Mean and 95th percentile of t(chosen)/t(best) - 1 over the rows."""
    if not rows:
        return {"mean": None, "p95": None, "max": None, "n": 0}
    reg = []
    for r, c in zip(rows, choices):
        t = np.array(r["times"], dtype=np.float64)
        reg.append(t[c] / np.nanmin(t) - 1.0)
    reg = np.array(reg)
    return {"mean": float(np.mean(reg)), "p95": float(np.percentile(reg, 95)), "max": float(np.max(reg)),
            "n": int(reg.size)}


def load_selector(params: np.ndarray) -> None:
    arr = np.ascontiguousarray(params, dtype=np.float32)
    st = B.strassen_selector_load(arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), arr.size)
    if st != 0:
        raise B.StrassenError(st, "strassen_selector_load")


def load_default_selector() -> Dict:
    """Load the network shipped with the package (trained on this library's timings on
    a GB300) into the library, enabled for the dtypes where it beat the analytic model
    on held-out shapes.  Returns the file's metadata."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "selector_gb300.json")
    with open(path) as fh:
        meta = json.load(fh)
    load_selector(np.array(meta["params"], dtype=np.float32))
    for d, on in meta["use_for_dtype"].items():
        st = B.strassen_selector_use(int(d), 1 if on else 0)
        if st != 0:
            raise B.StrassenError(st, "strassen_selector_use")
    return {k: v for k, v in meta.items() if k != "params"}


def save_rows(path: str, rows) -> None:
    with open(path, "w") as fh:
        json.dump(rows, fh)


def load_rows(spec: str):
    """Timed rows from a JSON list, or from a file of one JSON row per line (.jsonl).
    `spec` is a comma-separated list of such files, each optionally followed by
    ":f64" or ":oz_bf16" to keep only that dtype's rows (for example the FP64 rows of
    an earlier run together with freshly timed split-precision rows)."""
    names = {v: k for k, v in DTYPE_NAME.items()}
    rows = []
    for part in spec.split(","):
        path, _, want = part.partition(":")
        with open(path) as fh:
            got = [json.loads(line) for line in fh if line.strip()] if path.endswith(".jsonl") else json.load(fh)
        if want:
            if want not in names:
                raise ValueError("unknown dtype filter %r" % want)
            got = [r for r in got if r["dtype"] == names[want]]
        rows += got
    return rows


SWEEP_SQUARE = [2048 * i for i in range(1, 9)]
SWEEP_RANKK = [256, 512, 1024, 2048, 4096]
FIXED_RULES = {"always_1L_ABC": 2, "always_2L_ABC": 8, "always_3L_ABC": 14, "classical": 0}


def candidate_name(c: int) -> str:
    lv, var, tile = B.strassen_selector_candidate(c)
    if lv == 0:
        return f"classical/{128 if tile == 0 else 64}"
    return f"{lv}L {['ABC', 'AB', 'Naive'][var]}/{128 if tile == 0 else 64}"


def sweep(out_dir: str) -> List[Dict]:
    """The FP64 shape sweep: square m = n = k in 2048..16384 (step 2048) and rank-k
    m = n = 16384 with k in 256..4096, every candidate (levels 0-3, variants, tiles),
    effective GFLOP/s (2mnk/t); writes sweep_fp64.json and sweep_fp64.md into out_dir."""
    import os
    shapes = [(n, n, n) for n in SWEEP_SQUARE] + [(16384, 16384, k) for k in SWEEP_RANKK]
    timer = Timer(16384 * 16384, 16384 * 16384, 16384 * 16384)
    cs = [0] + [c for c in range(2, NC) if B.strassen_selector_candidate(c)[2] == 0]  # 128-wide tiles
    rows = measure(shapes, B.STRASSEN_F64, timer, cands=cs)
    names = [candidate_name(c) for c in cs]
    lines = ["| m | n | k | " + " | ".join(names) + " | best | best / classical |",
             "|" + "---|" * (len(names) + 5)]
    for r in rows:
        times = [r["times"][c] for c in cs]
        eff = [2.0 * r["m"] * r["n"] * r["k"] / t / 1e9 for t in times]
        b = int(np.nanargmin(np.array(times, dtype=np.float64)))
        lines.append(f"| {r['m']} | {r['n']} | {r['k']} | " + " | ".join(f"{v:.0f}" for v in eff) +
                     f" | {names[b]} | {eff[b] / eff[0]:.3f} |")
    os.makedirs(out_dir, exist_ok=True)
    save_rows(os.path.join(out_dir, "sweep_fp64.json"), rows)
    with open(os.path.join(out_dir, "sweep_fp64.md"), "w") as fh:
        fh.write("Effective GFLOP/s (2mnk/t), FP64, A, B, C uniform[-1,1], one GB300\n\n" + "\n".join(lines) + "\n")
    print("\n".join(lines))
    return rows


def evaluate(params, rows) -> Dict:
    """Regret of the network, the selection without it (analytic model / classical
    slices), the fixed rules and exhaustive timing on timed rows."""
    out = {"mlp": regret(rows, choose_mlp(params, rows)) if params is not None else None,
           "without_network": regret(rows, choose_model(rows))}
    for name, c in FIXED_RULES.items():
        out[name] = regret(rows, choose_fixed(rows, c))
    out["exhaustive"] = regret(rows, [best_of(r) for r in rows])
    counts = {}
    for r in rows:
        nm = candidate_name(best_of(r))
        counts[nm] = counts.get(nm, 0) + 1
    out["best_counts"] = counts
    return out


def main(argv=None) -> int:
    """Exhaustive timing of seeded random shapes (m, n, k log-uniform in [lo, hi]),
    selector training with the library's kernels and held-out evaluation; writes the
    timed rows, the parameters and a regret summary as JSON into --out.  Timed rows can
    be reused (--train-rows, --heldout-rows).  With --sweep, runs the FP64 shape sweep
    instead."""
    import argparse
    import os
    import sys
    import time
    ap = argparse.ArgumentParser(prog="python -m paper_1605_01078_gb300.tune")
    ap.add_argument("--train", type=int, default=250, help="FP64 training shapes (seed 1), 20 timings each")
    ap.add_argument("--heldout", type=int, default=1000, help="FP64 held-out shapes")
    ap.add_argument("--oz-train", type=int, default=100, help="split-precision training shapes (seed 3)")
    ap.add_argument("--oz-heldout", type=int, default=200, help="split-precision held-out shapes")
    ap.add_argument("--lo", type=int, default=256)
    ap.add_argument("--hi", type=int, default=16384)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", required=True)
    ap.add_argument("--sweep", action="store_true", help="run the FP64 shape sweep only")
    ap.add_argument("--measure-only", action="store_true", help="time the shapes and save the rows; no training")
    ap.add_argument("--train-rows", default=None,
                    help="timed training rows saved by earlier runs: file[:dtype][,file[:dtype]...] (JSON)")
    ap.add_argument("--heldout-rows", default=None, help="timed held-out rows, as --train-rows")
    ap.add_argument("--train-skip", type=int, default=0,
                    help="skip the first N FP64 training shapes (already timed), time the rest of --train")
    ap.add_argument("--oz-train-skip", type=int, default=0, help="the same for the split-precision training shapes")
    ap.add_argument("--ship", default=None,
                    help="also write the trained network in the shipped format (data/selector_gb300.json): "
                         "parameters, the held-out regrets, and the dtypes where it beat the method without it")
    ap.add_argument("--heldout-seed", type=int, default=2)
    ap.add_argument("--oz-heldout-seed", type=int, default=4)
    a = ap.parse_args(argv)
    if a.sweep:
        sweep(a.out)
        return 0
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import workloads as W
    os.makedirs(a.out, exist_ok=True)
    f64, oz = B.STRASSEN_F64, B.STRASSEN_F64_OZ_BF16
    timer = None
    t0 = time.time()

    def get_timer():
        nonlocal timer
        if timer is None:
            timer = Timer(a.hi * a.hi, a.hi * a.hi, a.hi * a.hi)
        return timer

    if a.train_rows:
        train_rows = load_rows(a.train_rows)
    else:
        log = os.path.join(a.out, "selector_train_rows.jsonl")
        train_rows = measure(W.loguniform_shapes(a.train, 1, a.lo, a.hi)[a.train_skip:], f64, get_timer(),
                             log_path=log)
        train_rows += measure(W.loguniform_shapes(a.oz_train, 3, a.lo, a.hi)[a.oz_train_skip:], oz, get_timer(),
                              log_path=log)
        save_rows(os.path.join(a.out, "selector_train_rows.json"), train_rows)
    t_train = time.time() - t0
    if a.heldout_rows:
        held = load_rows(a.heldout_rows)
    else:
        log = os.path.join(a.out, "selector_heldout_rows.jsonl")
        held = measure(W.loguniform_shapes(a.heldout, a.heldout_seed, a.lo, a.hi), f64, get_timer(), log_path=log)
        held += measure(W.loguniform_shapes(a.oz_heldout, a.oz_heldout_seed, a.lo, a.hi), oz, get_timer(),
                        log_path=log)
        save_rows(os.path.join(a.out, "selector_heldout_rows.json"), held)
    t_held = time.time() - t0 - t_train
    if a.measure_only:
        return 0
    params, hist = train(train_rows, steps=a.steps, lr=a.lr, seed=0)
    summary = {"timings_train": int(sum(np.isfinite(np.array(r["times"], dtype=float)).sum() for r in train_rows)),
               "shapes_train": len(train_rows), "seconds_measuring": [t_train, t_held], "loss_history": hist,
               "steps": a.steps, "lr": a.lr}
    for name, d in (("f64", f64), ("oz_bf16", oz)):
        rows = [r for r in held if r["dtype"] == d]
        summary[name] = evaluate(params, rows)
        summary[name]["shapes"] = len(rows)
    with open(os.path.join(a.out, "selector_params.json"), "w") as fh:
        json.dump([float(v) for v in params], fh)
    with open(os.path.join(a.out, "selector_summary.json"), "w") as fh:
        json.dump(summary, fh, indent=1)
    if a.ship:
        use = {}
        regrets = {}
        for name, d in (("f64", f64), ("oz_bf16", oz)):
            r_m, r_w = summary[name]["mlp"]["mean"], summary[name]["without_network"]["mean"]
            use[str(d)] = bool(r_m is not None and r_w is not None and r_m < r_w)
            regrets[name] = {"mlp": r_m, "without_network": r_w, "shapes": summary[name]["shapes"]}
        use.setdefault("1", False)
        meta = {"description": (
                    f"Variant-selector MLP ({B.SELECTOR_INPUTS}-64-64-{NC}, FP32) predicting a correction to the "
                    f"analytic model's log2 seconds, trained with the library's kernels ({a.steps} full-batch Adam "
                    f"steps, lr {a.lr}) on {summary['timings_train']} timings of {summary['shapes_train']} shapes "
                    f"(m, n, k log-uniform in [{a.lo}, {a.hi}]) measured on one GB300; held out: "
                    f"{regrets['f64']['shapes']} FP64 and {regrets['oz_bf16']['shapes']} split-precision shapes. "
                    "use_for_dtype: where its mean held-out regret is below the method without it."),
                "use_for_dtype": use, "heldout_regret_mean": regrets,
                "params": [float(v) for v in params]}
        with open(a.ship, "w") as fh:
            json.dump(meta, fh)
    print(json.dumps({k: summary[k] for k in ("f64", "oz_bf16")}, indent=1))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
