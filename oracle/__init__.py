"""CPU oracle for Strassen-fused GEMM (Huang, Smith, Henry, van de Geijn 2016).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU leg of ``bench.py`` (the CPU baseline and the exact and textbook entries behind its
error figures) may import this package.  It shares no code with the
CUDA library in ``paper_1605_01078_gb300`` and never imports it.

Contents
--------
* :func:`gemm`, :func:`strassen`, :func:`strassen_sampled`, :func:`gemm_sampled` --
  thin numpy wrappers over the plain C in ``oracle.c`` (classical definition, Section
  2.1; recursive textbook Strassen per Figure 1, Sections 3.1-3.3, in full or entry by
  entry; Dot2-compensated sampled entries).
* :func:`dgemm` -- alpha op(A) op(B) + beta C by that definition (Section 2.2).
* :func:`dsyrk` -- the symmetric rank-k update alpha op(A) op(A)^T + beta C on one
  triangle, by the same definition (a level-3 BLAS user of the method, Section 6).
* :mod:`oracle.tables` -- the one-level table of Figure 1 and the L-level tables of
  Eq. 4 built as Kronecker powers of it (Sections 3.5-3.6).
* :mod:`oracle.ozaki` -- error-free splitting of FP64 operands into integer slices
  and their exact products (split-precision emulation).
* :mod:`oracle.mlp` -- FP64 forward/backward of the variant-selector MLP.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with plain gcc (portable flags only:
    no -march, no contraction of a*b+c into fma, so that the arithmetic is exactly
    what the source says on x86_64 and aarch64 alike)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")
_omp = None


def build_timing(force: bool = False) -> str:
    """Compile the timing variant ``liboracle_omp.so``: the same source at -O3 with
    OpenMP (the rows of each classical product split over threads), still without
    contraction into fma, so every entry is computed exactly as in :func:`build`."""
    if force or not os.path.exists(_OMP_PATH) or (
            os.path.getmtime(_OMP_PATH) < os.path.getmtime(_SRC)):
        tmp = _OMP_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC])
        os.replace(tmp, _OMP_PATH)
    return _OMP_PATH


def host_cores() -> int:
    """Cores this process may run on (sched_getaffinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def strassen_timed(A: np.ndarray, B: np.ndarray, C: np.ndarray, levels: int, threads: int) -> int:
    """:func:`strassen` from the OpenMP timing build on ``threads`` threads (for timing
    the oracle on the host's cores; results equal :func:`strassen`'s)."""
    global _omp
    _check2d(A, "A"); _check2d(B, "B"); _check2d(C, "C")
    m, k = A.shape
    k2, n = B.shape
    if k2 != k or C.shape != (m, n):
        raise ValueError("shape mismatch")
    if _omp is None:
        build_timing()
        lib = ctypes.CDLL(_OMP_PATH)
        i64, dp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        lib.oracle_strassen.restype = i64
        lib.oracle_strassen.argtypes = [ctypes.c_int, i64, i64, i64, dp, i64, dp, i64, dp, i64]
        lib.omp_set_num_threads.restype = None
        lib.omp_set_num_threads.argtypes = [ctypes.c_int]
        _omp = lib
    _omp.omp_set_num_threads(int(threads))
    r = _omp.oracle_strassen(int(levels), m, n, k, _dp(A), A.strides[0] // 8, _dp(B), B.strides[0] // 8,
                             _dp(C), C.strides[0] // 8)
    if r < 0:
        raise MemoryError("oracle_strassen")
    return int(r)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, dp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        lib.oracle_gemm.restype = i64
        lib.oracle_gemm.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64]
        lib.oracle_strassen.restype = i64
        lib.oracle_strassen.argtypes = [ctypes.c_int, i64, i64, i64, dp, i64, dp, i64, dp, i64]
        lib.oracle_strassen_sampled.restype = ctypes.c_int
        lib.oracle_strassen_sampled.argtypes = [ctypes.c_int, i64, i64, i64, dp, i64, dp, i64, dp, i64,
                                                ctypes.POINTER(i64), ctypes.POINTER(i64), i64, dp]
        lib.oracle_gemm_sampled.restype = None
        lib.oracle_gemm_sampled.argtypes = [i64, dp, i64, dp, i64, dp, i64,
                                            ctypes.POINTER(i64), ctypes.POINTER(i64), i64, dp]
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check2d(x: np.ndarray, name: str) -> np.ndarray:
    if x.dtype != np.float64 or x.ndim != 2:
        raise TypeError(f"{name} must be a 2-D float64 array")
    if x.strides[1] != 8 or x.strides[0] % 8:
        raise TypeError(f"{name} must be row-major with unit column stride")
    return x


def gemm(A: np.ndarray, B: np.ndarray, C: np.ndarray) -> int:
    """In place: C += A @ B by the classical definition (Section 2.1).

    Returns the number of scalar multiplications (m*n*k)."""
    _check2d(A, "A"); _check2d(B, "B"); _check2d(C, "C")
    m, k = A.shape
    k2, n = B.shape
    if k2 != k or C.shape != (m, n):
        raise ValueError("shape mismatch")
    r = _load().oracle_gemm(m, n, k, _dp(A), A.strides[0] // 8, _dp(B), B.strides[0] // 8,
                            _dp(C), C.strides[0] // 8)
    if r < 0:
        raise MemoryError("oracle_gemm")
    return int(r)


def dgemm(transa: int, transb: int, alpha: float, A: np.ndarray, B: np.ndarray, beta: float,
          C: np.ndarray) -> np.ndarray:
    """The BLAS operation alpha op(A) op(B) + beta C (Section 2.2's DGEMM before its
    reduction to alpha = beta = 1), op(X) = X^T when trans is set: the product by the
    classical definition (:func:`gemm` on op(A), op(B)), then one scaling of it and of C
    and one addition per entry.  beta = 0 does not read C.  Returns a new array."""
    Aop = np.ascontiguousarray(A.T if transa else A, dtype=np.float64)
    Bop = np.ascontiguousarray(B.T if transb else B, dtype=np.float64)
    P = np.zeros((Aop.shape[0], Bop.shape[1]))
    if Aop.shape[1] > 0:
        gemm(Aop, Bop, P)
    base = np.zeros_like(P) if beta == 0 else beta * np.asarray(C, dtype=np.float64)
    return base + alpha * P


def dsyrk(uplo: int, trans: int, alpha: float, A: np.ndarray, beta: float, C: np.ndarray) -> np.ndarray:
    """The BLAS symmetric rank-k update on one triangle (a level-3 BLAS operation the
    paper's conclusion lists among the users of the same Strassen approach):
    op(A) = A (n x k) for trans = 0, A^T for trans = 1 (A stored k x n); P = op(A) op(A)^T
    by the classical definition (:func:`gemm`); then for uplo = 0 every entry with
    j <= i (lower triangle, diagonal included), for uplo = 1 every entry with j >= i,
    becomes alpha P_ij + beta C_ij (beta = 0 does not read C), and the rest of C is
    returned unchanged.  Returns a new array."""
    Aop = np.ascontiguousarray(A.T if trans else A, dtype=np.float64)
    n = Aop.shape[0]
    P = np.zeros((n, n))
    if Aop.shape[1] > 0:
        gemm(Aop, np.ascontiguousarray(Aop.T), P)
    out = np.array(C, dtype=np.float64, copy=True)
    i, j = np.indices((n, n))
    tri = (j <= i) if uplo == 0 else (j >= i)
    base = np.zeros_like(P) if beta == 0 else beta * out
    out[tri] = (base + alpha * P)[tri]
    return out


def strassen(A: np.ndarray, B: np.ndarray, C: np.ndarray, levels: int) -> int:
    """In place: C += A @ B by ``levels`` recursive levels of Figure 1 (textbook
    Strassen with zero padding of odd sizes), classical at the leaves.

    Returns the number of scalar multiplications performed at the leaves
    (7^L * ceil-halved sizes, against m*n*k for the classical definition)."""
    _check2d(A, "A"); _check2d(B, "B"); _check2d(C, "C")
    m, k = A.shape
    k2, n = B.shape
    if k2 != k or C.shape != (m, n):
        raise ValueError("shape mismatch")
    r = _load().oracle_strassen(int(levels), m, n, k, _dp(A), A.strides[0] // 8,
                                _dp(B), B.strides[0] // 8, _dp(C), C.strides[0] // 8)
    if r < 0:
        raise MemoryError("oracle_strassen")
    return int(r)


def gemm_sampled(A: np.ndarray, B: np.ndarray, C0: np.ndarray | None,
                 rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Entries (rows[t], cols[t]) of C0 + A @ B, each computed with the compensated
    dot product Dot2 (twice-working-precision accuracy, then rounded)."""
    _check2d(A, "A"); _check2d(B, "B")
    m, k = A.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    if rows.shape != cols.shape or rows.ndim != 1:
        raise ValueError("rows/cols must be 1-D of equal length")
    if rows.size and (rows.min() < 0 or rows.max() >= m or cols.min() < 0 or cols.max() >= B.shape[1]):
        raise IndexError("sample index out of range")
    out = np.empty(rows.size, dtype=np.float64)
    if C0 is not None:
        _check2d(C0, "C0")
        c0p, ldc = _dp(C0), C0.strides[0] // 8
    else:
        c0p, ldc = ctypes.cast(None, ctypes.POINTER(ctypes.c_double)), 0
    P64 = ctypes.POINTER(ctypes.c_int64)
    _load().oracle_gemm_sampled(k, _dp(A), A.strides[0] // 8, _dp(B), B.strides[0] // 8,
                                c0p, ldc, rows.ctypes.data_as(P64), cols.ctypes.data_as(P64),
                                rows.size, _dp(out))
    return out


def strassen_sampled(A: np.ndarray, B: np.ndarray, C0: np.ndarray | None, rows: np.ndarray,
                     cols: np.ndarray, levels: int) -> np.ndarray:
    """Entries (rows[t], cols[t]) of the result :func:`strassen` would leave in a copy
    of C0 (zeros when None), computed one entry at a time in exactly its order of
    operations (bit for bit the same values), for products too large for the full
    recursion on a CPU."""
    _check2d(A, "A"); _check2d(B, "B")
    m, k = A.shape
    k2, n = B.shape
    if k2 != k:
        raise ValueError("shape mismatch")
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    if rows.shape != cols.shape or rows.ndim != 1:
        raise ValueError("rows/cols must be 1-D of equal length")
    if rows.size and (rows.min() < 0 or rows.max() >= m or cols.min() < 0 or cols.max() >= n):
        raise IndexError("sample index out of range")
    Bt = np.ascontiguousarray(B.T)
    out = np.empty(rows.size, dtype=np.float64)
    if C0 is not None:
        _check2d(C0, "C0")
        c0p, ldc = _dp(C0), C0.strides[0] // 8
    else:
        c0p, ldc = ctypes.cast(None, ctypes.POINTER(ctypes.c_double)), 0
    P64 = ctypes.POINTER(ctypes.c_int64)
    r = _load().oracle_strassen_sampled(int(levels), m, n, k, _dp(A), A.strides[0] // 8, _dp(Bt), k,
                                        c0p, ldc, rows.ctypes.data_as(P64), cols.ctypes.data_as(P64),
                                        rows.size, _dp(out))
    if r < 0:
        raise MemoryError("oracle_strassen_sampled")
    return out


def max_rel_err(C: np.ndarray, C_ref: np.ndarray, A: np.ndarray, B: np.ndarray) -> float:
    """Element-wise max-norm error scaled by the operands: max|C - C_ref| /
    (max|A| * max|B|).  Zero operands give the plain max error."""
    den = float(np.max(np.abs(A), initial=0.0)) * float(np.max(np.abs(B), initial=0.0))
    err = float(np.max(np.abs(np.asarray(C) - np.asarray(C_ref)), initial=0.0))
    return err / den if den > 0 else err


__all__ = ["build", "build_timing", "host_cores", "gemm", "dgemm", "dsyrk", "strassen", "strassen_timed", "strassen_sampled",
           "gemm_sampled", "max_rel_err"]
