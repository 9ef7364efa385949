"""SUMMA across GPUs with local Strassen rank-b updates (the distributed-memory
experiments of the paper's Section 5: a 2-D grid of processes, each broadcast step
followed by a local rank-b update with one- or two-level ABC Strassen).

Layout: a pr x pc process grid, rank = row * pc + col.  C (m x n) is split into pr x pc
blocks, A (m x k) into pr x pc blocks and B (k x n) into pr x pc blocks, with the block
boundaries of `block_ranges`; rank (i, j) holds A_ij, B_ij and C_ij.  For every panel of
b columns of A (= b rows of B), in order along k:

* the process column that owns the panel broadcasts its part of A's panel along each
  process row (the rows of A_i:, width b);
* the process row that owns the panel broadcasts its part of B's panel along each
  process column (the columns of B_:j, height b);
* every rank adds A_panel(i) B_panel(j) into C_ij by the local update, which by default
  is `strassen_gemm` on the rank's GPU (ABC Strassen, `levels` levels, rank-b update).

The broadcasts go through `torch.distributed` (NCCL on GPUs, gloo on CPUs) into each
rank's own memory; nothing here reads another GPU's memory directly.  The local update
is a parameter so that the panel logic can be exercised on CPU ranks with any exact
product (the tests pass one); with the default it runs only on CUDA tensors and raises
otherwise.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence, Tuple


def block_ranges(extent: int, parts: int) -> List[Tuple[int, int]]:
    """[begin, end) of each of `parts` nearly equal blocks of `extent` (the first
    extent % parts blocks one longer)."""
    if parts <= 0:
        raise ValueError("parts must be positive")
    base, extra = divmod(extent, parts)
    out, b = [], 0
    for p in range(parts):
        e = b + base + (1 if p < extra else 0)
        out.append((b, e))
        b = e
    return out


def panel_plan(k: int, pc: int, pr: int, b: int) -> List[Tuple[int, int, int, int, int, int]]:
    """The panels of the k dimension in order: (k0, k1, owner column of A's part,
    offset inside that column's A block, owner row of B's part, offset inside that row's
    B block).  A panel never crosses a block boundary of either partition."""
    if b <= 0:
        raise ValueError("panel width must be positive")
    a_cols = block_ranges(k, pc)
    b_rows = block_ranges(k, pr)
    cuts = sorted({0, k} | {e for _, e in a_cols} | {e for _, e in b_rows})
    plan = []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        for k0 in range(lo, hi, b):
            k1 = min(k0 + b, hi)
            ja = next(j for j, (s, e) in enumerate(a_cols) if s <= k0 < e)
            ib = next(i for i, (s, e) in enumerate(b_rows) if s <= k0 < e)
            plan.append((k0, k1, ja, k0 - a_cols[ja][0], ib, k0 - b_rows[ib][0]))
    return plan


def strassen_update(levels: int = 1) -> Callable:
    """The default local update: C += A B on the rank's GPU with `levels` levels of ABC
    Strassen (strassen_gemm through the library)."""
    from . import gemm

    def update(A, B, C):
        if not (A.is_cuda and B.is_cuda and C.is_cuda):
            raise TypeError("the Strassen local update runs on CUDA tensors")
        gemm(A, B, C, levels=levels, variant="ABC")

    return update


def summa(A_local, B_local, C_local, m: int, n: int, k: int, grid: Tuple[int, int], b: int = 1024,
          update: Optional[Callable] = None, levels: int = 1, dist=None, row_groups: Optional[Sequence] = None,
          col_groups: Optional[Sequence] = None) -> None:
    """C_local += (A B)_ij on rank (i, j) of a pr x pc grid (see the module docstring).

    A_local, B_local, C_local: this rank's blocks (torch tensors, row-major, on the
    rank's device).  row_groups[i] / col_groups[j] are the process groups of process row
    i and process column j (as made by `make_groups`; every rank must pass the same
    lists).  update(A_panel, B_panel, C) performs C += A_panel B_panel.
    """
    import torch
    if dist is None:
        import torch.distributed as dist
    pr, pc = grid
    rank = dist.get_rank()
    if dist.get_world_size() != pr * pc:
        raise ValueError("the grid does not match the world size")
    i, j = divmod(rank, pc)
    rows, cols = block_ranges(m, pr), block_ranges(n, pc)
    mi, nj = rows[i][1] - rows[i][0], cols[j][1] - cols[j][0]
    a_cols, b_rows = block_ranges(k, pc), block_ranges(k, pr)
    if tuple(A_local.shape) != (mi, a_cols[j][1] - a_cols[j][0]) or \
            tuple(B_local.shape) != (b_rows[i][1] - b_rows[i][0], nj) or tuple(C_local.shape) != (mi, nj):
        raise ValueError("local blocks do not match the grid partition")
    if update is None:
        update = strassen_update(levels)
    for (k0, k1, ja, oa, ib, ob) in panel_plan(k, pc, pr, b):
        w = k1 - k0
        Ap = torch.empty((mi, w), dtype=A_local.dtype, device=A_local.device)
        Bp = torch.empty((w, nj), dtype=B_local.dtype, device=B_local.device)
        if j == ja:
            Ap.copy_(A_local[:, oa:oa + w])
        if i == ib:
            Bp.copy_(B_local[ob:ob + w, :])
        # along the process row i from column ja; along the process column j from row ib
        dist.broadcast(Ap, src=i * pc + ja, group=row_groups[i] if row_groups is not None else None)
        dist.broadcast(Bp, src=ib * pc + j, group=col_groups[j] if col_groups is not None else None)
        update(Ap, Bp, C_local)


def make_groups(grid: Tuple[int, int], dist=None):
    """The process groups of every process row and every process column of the grid
    (collective: every rank calls it with the same grid)."""
    if dist is None:
        import torch.distributed as dist
    pr, pc = grid
    row_groups = [dist.new_group([i * pc + j for j in range(pc)]) for i in range(pr)]
    col_groups = [dist.new_group([i * pc + j for i in range(pr)]) for j in range(pc)]
    return row_groups, col_groups
