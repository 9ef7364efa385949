"""SUMMA with local rank-b updates (the paper's distributed-memory form, Section 5).

CPU tests: the panel plan and block partition, and the whole exchange on 2 and 4 gloo
ranks (1 x 2, 2 x 1 and 2 x 2 grids) with an exact local product (the oracle's classical
definition) on integer inputs, so the assembled C must equal the full product bit for
bit.  GPU test: one rank over NCCL with the library's Strassen update (the only
multi-process configuration a one-GPU run can hold).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1605_01078_gb300 import summa  # noqa: E402


def test_block_ranges_cover_the_extent():
    for extent, parts in ((10, 3), (7, 7), (5, 8), (0, 2), (1024, 4)):
        r = summa.block_ranges(extent, parts)
        assert len(r) == parts and r[0][0] == 0 and r[-1][1] == extent
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        assert max(e - s for s, e in r) - min(e - s for s, e in r) <= 1


def test_panel_plan_splits_k_at_both_partitions():
    k, pc, pr, b = 1000, 3, 2, 128
    plan = summa.panel_plan(k, pc, pr, b)
    assert plan[0][0] == 0 and plan[-1][1] == k
    assert all(p[1] == q[0] for p, q in zip(plan, plan[1:]))
    a_cols, b_rows = summa.block_ranges(k, pc), summa.block_ranges(k, pr)
    for k0, k1, ja, oa, ib, ob in plan:
        assert 0 < k1 - k0 <= b
        assert a_cols[ja][0] <= k0 and k1 <= a_cols[ja][1] and oa == k0 - a_cols[ja][0]
        assert b_rows[ib][0] <= k0 and k1 <= b_rows[ib][1] and ob == k0 - b_rows[ib][0]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _exact_update(A, B, C):
    import oracle
    oracle.gemm(np.ascontiguousarray(A.numpy()), np.ascontiguousarray(B.numpy()), C.numpy())


def _worker(rank, world, port, grid, shape, b, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import workloads as W
        m, n, k = shape
        A, B, C = W.integer(m, k, 1), W.integer(k, n, 2), W.integer(m, n, 3)
        pr, pc = grid
        i, j = divmod(rank, pc)
        rows, cols = summa.block_ranges(m, pr), summa.block_ranges(n, pc)
        ka, kb = summa.block_ranges(k, pc), summa.block_ranges(k, pr)
        A_l = torch.from_numpy(np.ascontiguousarray(A[rows[i][0]:rows[i][1], ka[j][0]:ka[j][1]]))
        B_l = torch.from_numpy(np.ascontiguousarray(B[kb[i][0]:kb[i][1], cols[j][0]:cols[j][1]]))
        C_l = torch.from_numpy(np.ascontiguousarray(C[rows[i][0]:rows[i][1], cols[j][0]:cols[j][1]]))
        rg, cg = summa.make_groups(grid)
        summa.summa(A_l, B_l, C_l, m, n, k, grid, b=b, update=_exact_update, row_groups=rg, col_groups=cg)
        out[rank] = C_l.numpy().copy()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("grid,shape,b", [((1, 2), (37, 29, 53), 8), ((2, 1), (40, 33, 31), 16),
                                          ((2, 2), (45, 38, 61), 7)])
def test_summa_on_gloo_ranks_equals_the_full_product(grid, shape, b):
    import oracle
    import workloads as W
    world = grid[0] * grid[1]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), grid, shape, b, out), nprocs=world, join=True)
        res = dict(out)
    m, n, k = shape
    A, B, C = W.integer(m, k, 1), W.integer(k, n, 2), W.integer(m, n, 3)
    ref = C.copy()
    oracle.gemm(A, B, ref)
    rows, cols = summa.block_ranges(m, grid[0]), summa.block_ranges(n, grid[1])
    for rank, blk in res.items():
        i, j = divmod(rank, grid[1])
        assert np.array_equal(blk, ref[rows[i][0]:rows[i][1], cols[j][0]:cols[j][1]])


def test_summa_rejects_a_mismatched_grid():
    class FakeDist:
        @staticmethod
        def get_rank():
            return 0

        @staticmethod
        def get_world_size():
            return 3

    t = torch.zeros((2, 2), dtype=torch.float64)
    with pytest.raises(ValueError):
        summa.summa(t, t, t, 2, 2, 2, (2, 2), dist=FakeDist)


@pytest.mark.gpu
def test_summa_one_gpu_rank_with_the_strassen_update():
    """One NCCL rank (1 x 1 grid): every panel goes through the library's two-level ABC
    update; integer inputs give the oracle's product bit for bit."""
    import oracle
    import workloads as W
    store = dist.HashStore()
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", store=store, rank=0, world_size=1)
    try:
        m, n, k = 700, 520, 900
        A, B, C = W.integer(m, k, 4), W.integer(k, n, 5), W.integer(m, n, 6)
        dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C))
        summa.summa(dA, dB, dC, m, n, k, (1, 1), b=256, levels=2)
        torch.cuda.synchronize()
        ref = C.copy()
        oracle.gemm(A, B, ref)
        assert np.array_equal(dC.cpu().numpy(), ref)
    finally:
        dist.destroy_process_group()
