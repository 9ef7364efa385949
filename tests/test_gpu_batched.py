"""The batched persistent launch (many uneven problems in one kernel launch) against
the oracle, its capture in a CUDA graph, and the bounded device-side wait."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1605_01078_gb300 as sg
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 1e-13, 2: 1e-12, 3: 1e-12}


def problems_array(items):
    arr = (sg.strassen_problem * len(items))()
    for i, (A, B, C, levels, variant) in enumerate(items):
        m, k = A.shape
        n = B.shape[1]
        arr[i] = sg.strassen_problem(m, n, k, A.data_ptr(), B.data_ptr(), C.data_ptr(),
                                     A.stride(0), B.stride(0), C.stride(0), levels, variant)
    return arr


def test_batched_integer_bit_exact_mixed_levels():
    shapes = W.loguniform_shapes(40, seed=3, lo=1, hi=300)
    items, host = [], []
    for i, (m, n, k) in enumerate(shapes):
        A, B, C = W.integer(m, k, 10 * i), W.integer(k, n, 10 * i + 1), W.integer(m, n, 10 * i + 2)
        ref = C.copy()
        oracle.gemm(A, B, ref)
        dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C))
        items.append((dA, dB, dC, i % 4, sg.STRASSEN_ABC))
        host.append(ref)
    arr = problems_array(items)
    st = sg.strassen_gemm_batched(len(items), arr, sg.STRASSEN_F64, torch.cuda.current_stream().cuda_stream)
    assert st == 0, sg.strassen_status_string(st)
    torch.cuda.synchronize()
    for (dA, dB, dC, lv, _), ref in zip(items, host):
        assert np.array_equal(dC.cpu().numpy(), ref), (tuple(dA.shape), tuple(dB.shape), lv)


def test_batched_large_aligned_problems_bit_exact():
    """Large tile-aligned problems (the launch takes the 128-wide tile) mixed over
    levels 0..3, integer inputs: bit for bit against the oracle."""
    shapes = [(1536, 1024, 512), (1024, 1536, 768), (2048, 1024, 256), (1024, 1024, 1024)]
    items, host = [], []
    for i, (m, n, k) in enumerate(shapes):
        A, B, C = W.integer(m, k, 70 + i), W.integer(k, n, 80 + i), W.integer(m, n, 90 + i)
        ref = C.copy()
        oracle.gemm(A, B, ref)
        items.append(tuple(torch.from_numpy(x).cuda() for x in (A, B, C)) + (i, sg.STRASSEN_ABC))
        host.append(ref)
    arr = problems_array(items)
    assert sg.strassen_gemm_batched(len(items), arr, sg.STRASSEN_F64, torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    for it, ref in zip(items, host):
        assert np.array_equal(it[2].cpu().numpy(), ref)


def test_batched_rejects_overlapping_outputs_and_bad_problems():
    A = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    B = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    C = torch.zeros((16, 8), dtype=torch.float64, device="cuda")
    arr = problems_array([(A, B, C[:8], 1, 0), (A, B, C[4:12], 1, 0)])
    assert sg.strassen_gemm_batched(2, arr, 0, 0) == -9
    arr = problems_array([(A, B, C[:8], 4, 0)])
    assert sg.strassen_gemm_batched(1, arr, 0, 0) == -4
    assert sg.strassen_gemm_batched(-1, arr, 0, 0) == -9
    assert sg.strassen_gemm_batched(0, None, 0, 0) == 0
    assert sg.strassen_gemm_batched(1, None, 0, 0) == -3


def test_batched_captured_in_a_cuda_graph():
    shapes = [(200, 130, 90), (64, 64, 64), (300, 17, 129), (5, 7, 3)]
    items, refs = [], []
    for i, (m, n, k) in enumerate(shapes):
        A, B, C = W.integer(m, k, 50 + i), W.integer(k, n, 60 + i), W.integer(m, n, 70 + i)
        ref = C.copy()
        oracle.gemm(A, B, ref)
        oracle.gemm(A, B, ref)  # two replays: C + 2 AB
        items.append(tuple(torch.from_numpy(x).cuda() for x in (A, B, C)) + (1 + i % 2, 0))
        refs.append(ref)
    arr = problems_array(items)
    # one uncaptured call first: the library sets up its per-device state
    scratch = [torch.zeros_like(it[2]) for it in items]
    warm = problems_array([(it[0], it[1], s, it[3], 0) for it, s in zip(items, scratch)])
    assert sg.strassen_gemm_batched(len(items), warm, 0, torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        st = sg.strassen_gemm_batched(len(items), arr, 0, torch.cuda.current_stream().cuda_stream)
    assert st == 0
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for it, ref in zip(items, refs):
        assert np.array_equal(it[2].cpu().numpy(), ref)


def test_batched_256_uneven_problems_sampled():
    """256 problems, m, n, k log-uniform in [256, 4096] (seed 0), levels from the
    selector, one launch; 16 entries per problem checked against Dot2."""
    shapes = W.loguniform_shapes(256, seed=0, lo=256, hi=4096)
    items = []
    for i, (m, n, k) in enumerate(shapes):
        A = W.uniform_device(m, k, 1000 + i)
        B = W.uniform_device(k, n, 2000 + i)
        C = W.uniform_device(m, n, 3000 + i)
        items.append((A, B, C, C.clone(), -1))
    arr = problems_array([(A, B, C, lv, sg.STRASSEN_AUTO) for (A, B, C, _, lv) in items])
    st = sg.strassen_gemm_batched(len(items), arr, 0, torch.cuda.current_stream().cuda_stream)
    assert st == 0, sg.strassen_status_string(st)
    torch.cuda.synchronize()
    for i, (A, B, C, C0, _) in enumerate(items):
        m, k = A.shape
        n = B.shape[1]
        rows, cols = W.sample_indices(m, n, 16, 500 + i)
        Ar = A[torch.from_numpy(rows).cuda()].cpu().numpy()
        Bc = B[:, torch.from_numpy(cols).cuda()].cpu().numpy()
        c0 = C0.cpu().numpy()[rows, cols]
        ref = np.array([oracle.gemm_sampled(Ar[t:t + 1], np.ascontiguousarray(Bc[:, t:t + 1]), None,
                                            np.array([0]), np.array([0]))[0] for t in range(16)]) + c0
        got = C.cpu().numpy()[rows, cols]
        lv, _, _ = sg.strassen_select(m, n, k, 0)
        den = float(torch.max(torch.sum(torch.abs(A), dim=1))) * float(torch.max(torch.abs(B)))
        assert float(np.max(np.abs(got - ref))) / den <= TOL[lv], (i, m, n, k)


def test_bounded_wait_reports_timeout_and_context_survives():
    s = torch.cuda.current_stream().cuda_stream
    assert sg.strassen_device_status(s) == 0
    assert sg.strassen_check_wait_timeout(2_000_000, s) == 0   # about 1 ms of SM clock
    assert sg.strassen_device_status(s) == -7
    assert sg.strassen_device_status(s) == 0                    # cleared on read
    assert sg.strassen_check_wait_timeout(-1, s) == -9
    A, B = W.integer(33, 21, 1), W.integer(21, 17, 2)
    dC = torch.zeros((33, 17), dtype=torch.float64, device="cuda")
    sg.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), dC, levels=1, variant="ABC")
    torch.cuda.synchronize()
    assert np.array_equal(dC.cpu().numpy(), A @ B)
    assert sg.strassen_device_status(s) == 0


def test_integer_pipe_addition_matches_dadd_on_the_device():
    """The staging kernels form operand sums with an integer-pipe binary64 addition;
    on the GPU it must agree bitwise with the hardware FP64 addition."""
    assert sg.strassen_check_int_fadd(1 << 24, 12345) == 0
    assert sg.strassen_check_int_fadd(1 << 20, 999) == 0
