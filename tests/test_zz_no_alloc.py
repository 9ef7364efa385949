"""strassen_gemm_ab_noalloc against strassen_gemm(..., STRASSEN_AB, ...) on the GPU.

The no-allocation entry point exists for callers that cannot allocate device memory
while they run (a process whose memory belongs to its own pooling allocator, a
latency-bound loop where an allocation could synchronise the device, code with no
out-of-memory path).  Its temporary lives in one fixed array inside the library that
keeps the previous call's contents, so every case here makes two calls in a row and
checks both against the regular AB entry point: bit for bit on integer-valued inputs,
and within the float tolerance the other GPU tests use (1e-13 at one level, 1e-12 at
two and three, max|C1 - C2| / (max|A| max|B|)) on uniform[-1, 1] inputs.

This file is collected last on purpose; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1605_01078_gb300 as sg
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {1: 1e-13, 2: 1e-12, 3: 1e-12}
SCRATCH_ELEMS = 1 << 22  # doubles in the library's fixed array


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def regular_ab(A, B, C0, levels):
    C = C0.clone()
    m, k = A.shape
    n = B.shape[1]
    st = sg.strassen_gemm(m, n, k, A.data_ptr(), k, B.data_ptr(), n, C.data_ptr(), n, levels,
                          sg.STRASSEN_AB, sg.STRASSEN_F64, torch.cuda.current_stream().cuda_stream)
    assert st == 0, sg.strassen_status_string(st)
    return C


def no_alloc(A, B, C0, levels):
    C = C0.clone()
    m, k = A.shape
    n = B.shape[1]
    st = sg.strassen_gemm_ab_noalloc(m, n, k, A.data_ptr(), k, B.data_ptr(), n, C.data_ptr(), n, levels,
                                     torch.cuda.current_stream().cuda_stream)
    assert st == 0, sg.strassen_status_string(st)
    return C


def strict(C, R, A, B):
    den = float(torch.max(torch.abs(A))) * float(torch.max(torch.abs(B)))
    return float(torch.max(torch.abs(C - R))) / den


CASES = [
    # (m, n, k, levels, integer inputs)
    (13, 7, 11, 1, True),
    (300, 257, 129, 2, True),
    (1000, 999, 1001, 1, False),
    (1024, 1024, 1024, 2, False),
    (8192, 8192, 96, 2, True),   # M uses the whole array: (8192/4)^2 = 4 Mi doubles
    (301, 203, 150, 3, True),
]


@pytest.mark.parametrize("m,n,k,levels,integer", CASES)
def test_no_alloc_matches_ab_two_calls_in_a_row(m, n, k, levels, integer):
    gen = W.integer if integer else W.uniform
    A, B, C0 = dev(gen(m, k, 1)), dev(gen(k, n, 2)), dev(gen(m, n, 3))
    ref = regular_ab(A, B, C0, levels)
    for _ in range(2):
        got = no_alloc(A, B, C0, levels)
        torch.cuda.synchronize()
        if integer:
            assert torch.equal(got, ref)
        else:
            assert strict(got, ref, A, B) <= TOL[levels]


def test_no_alloc_after_a_larger_call_is_unaffected():
    """The array keeps the previous call's contents: a small call after a large one
    (and the reverse) must still match the regular entry point."""
    big = [dev(W.uniform(2000, 1500, 4)), dev(W.uniform(1500, 2100, 5)), dev(W.uniform(2000, 2100, 6))]
    small = [dev(W.integer(41, 37, 7)), dev(W.integer(37, 29, 8)), dev(W.integer(41, 29, 9))]
    for A, B, C0 in (big, small, big, small):
        got = no_alloc(A, B, C0, 1)
        ref = regular_ab(A, B, C0, 1)
        torch.cuda.synchronize()
        assert strict(got, ref, A, B) <= TOL[1]


def test_no_alloc_rejects_products_beyond_the_array():
    m = n = 4098            # one level: M would be 2049 x 2049 > 4 Mi doubles
    k = 8
    A = torch.zeros((m, k), dtype=torch.float64, device="cuda")
    B = torch.zeros((k, n), dtype=torch.float64, device="cuda")
    C = torch.full((m, n), 5.0, dtype=torch.float64, device="cuda")
    assert 2049 * 2049 > SCRATCH_ELEMS
    st = sg.strassen_gemm_ab_noalloc(m, n, k, A.data_ptr(), k, B.data_ptr(), n, C.data_ptr(), n, 1,
                                     torch.cuda.current_stream().cuda_stream)
    assert st == -10, sg.strassen_status_string(st)
    torch.cuda.synchronize()
    assert torch.all(C == 5.0)
    assert sg.strassen_gemm_ab_noalloc(m, n, k, A.data_ptr(), k, B.data_ptr(), n, C.data_ptr(), n, 4, 0) == -4


def _cudart():
    """The CUDA runtime the library is linked against (found among the loaded objects)."""
    sg.load_library()
    paths = []
    with open("/proc/self/maps") as fh:
        for line in fh:
            path = line.split()[-1]
            if "libcudart.so" in path and path not in paths:
                paths.append(path)
    if not paths:
        pytest.skip("no CUDA runtime among the loaded objects")
    return ctypes.CDLL(paths[0])


def test_no_alloc_call_makes_no_device_allocation():
    """The library's temporaries come from the device's current memory pool
    (cudaMallocAsync).  With the pool's high-water mark reset before each call, a
    no-allocation call must leave it at the memory in use before the call, while the
    regular AB call must raise it by at least its temporary M (so the probe does see the
    library's allocations)."""
    rt = _cudart()
    USED_CURRENT, USED_HIGH = 0x7, 0x8  # cudaMemPoolAttrUsedMemCurrent / UsedMemHigh
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetMemPool(ctypes.byref(pool), ctypes.c_int(torch.cuda.current_device())) == 0

    def attr(a):
        v = ctypes.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, ctypes.c_int(a), ctypes.byref(v)) == 0
        return v.value

    def reset_high():
        zero = ctypes.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, ctypes.c_int(USED_HIGH), ctypes.byref(zero)) == 0

    m = n = k = 1536
    A, B, C0 = dev(W.uniform(m, k, 11)), dev(W.uniform(k, n, 12)), dev(W.uniform(m, n, 13))
    no_alloc(A, B, C0, 1)  # first call on this device: its set-up
    for levels in (1, 2):
        torch.cuda.synchronize()
        before = attr(USED_CURRENT)
        reset_high()
        got = no_alloc(A, B, C0, levels)
        torch.cuda.synchronize()
        assert attr(USED_HIGH) == before, "the no-allocation call allocated from the pool"
        reset_high()
        ref = regular_ab(A, B, C0, levels)
        torch.cuda.synchronize()
        h = -(-m // 2 ** levels)
        assert attr(USED_HIGH) >= before + 8 * h * h, "the probe did not see the regular call's temporary"
        assert strict(got, ref, A, B) <= TOL[levels]
