"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the method: it only draws matrices and shapes.  All
draws use numpy's Philox bit generator keyed by the seed, so the same seed gives the
same matrices on x86_64 and aarch64 hosts.  Workload recipes (the paper uses no
dataset; its experiments use square, fixed-k and rank-k shapes of random matrices):

* ``uniform``  -- i.i.d. uniform[lo, hi) FP64 entries (default [-1, 1)).
* ``integer``  -- i.i.d. integers in [lo, hi] stored as FP64 (default {-4..4}): every
  sum and product of the Strassen path stays exactly representable.
* ``scaled``   -- u * 2^round(N(0, sigma)) with u uniform[-1, 1): entries spread over
  many binades, for the split-precision (Ozaki) error study.
* ``loguniform_shapes`` -- (m, n, k) triples with each size log-uniform in [lo, hi].
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def uniform(rows: int, cols: int, seed: int, lo: float = -1.0, hi: float = 1.0, ld: int | None = None) -> np.ndarray:
    """rows x cols FP64 matrix; with ``ld`` > cols it is a view into a rows x ld buffer
    whose padding columns hold NaN (so a kernel that reads them shows it)."""
    g = _rng(seed)
    x = g.uniform(lo, hi, size=(rows, cols))
    if ld is None or ld == cols:
        return np.ascontiguousarray(x)
    buf = np.full((rows, ld), np.nan)
    buf[:, :cols] = x
    return buf[:, :cols]


def integer(rows: int, cols: int, seed: int, lo: int = -4, hi: int = 4, ld: int | None = None) -> np.ndarray:
    g = _rng(seed)
    x = g.integers(lo, hi + 1, size=(rows, cols)).astype(np.float64)
    if ld is None or ld == cols:
        return np.ascontiguousarray(x)
    buf = np.full((rows, ld), np.nan)
    buf[:, :cols] = x
    return buf[:, :cols]


def scaled(rows: int, cols: int, seed: int, sigma: float) -> np.ndarray:
    g = _rng(seed)
    u = g.uniform(-1.0, 1.0, size=(rows, cols))
    e = np.rint(g.normal(0.0, sigma, size=(rows, cols))) if sigma > 0 else np.zeros((rows, cols))
    return np.ldexp(u, e.astype(np.int64))


def loguniform_shapes(count: int, seed: int, lo: int, hi: int) -> List[Tuple[int, int, int]]:
    g = _rng(seed)
    x = np.exp(g.uniform(np.log(lo), np.log(hi), size=(count, 3)))
    x = np.clip(np.rint(x).astype(np.int64), lo, hi)
    return [tuple(int(v) for v in row) for row in x]


def sample_indices(rows: int, cols: int, count: int, seed: int) -> Tuple[np.ndarray, np.ndarray]:
    """``count`` (row, col) positions, always including the four corners."""
    g = _rng(seed)
    r = g.integers(0, rows, size=count)
    c = g.integers(0, cols, size=count)
    r[:4] = [0, 0, rows - 1, rows - 1]
    c[:4] = [0, cols - 1, 0, cols - 1]
    return r.astype(np.int64), c.astype(np.int64)


def uniform_device(rows: int, cols: int, seed: int, device="cuda", lo: float = -1.0, hi: float = 1.0):
    """rows x cols FP64 uniform[lo, hi) drawn on the device by torch's generator
    (for workloads too large to draw on the host); the same seed gives the same
    matrix on the same device type."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    x = torch.rand((rows, cols), generator=g, dtype=torch.float64, device=device)
    return x.mul_(hi - lo).add_(lo)
