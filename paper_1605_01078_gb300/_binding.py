"""ctypes binding of the C ABI in ``include/strassen.h``.

Argument marshalling only: every function here forwards to the entry point of the
same name in ``libstrassen_gb300.so``; all arithmetic runs in the library's CUDA
kernels.  There is no CPU fallback: if the library cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstrassen_gb300.so")

# enums of strassen.h
STRASSEN_ABC, STRASSEN_AB, STRASSEN_NAIVE, STRASSEN_AUTO, STRASSEN_HYBRID = 0, 1, 2, 3, 4
STRASSEN_F64, STRASSEN_F64_OZ_INT8, STRASSEN_F64_OZ_BF16 = 0, 1, 2
STRASSEN_FLAG_DETERMINISTIC = 1
MAX_LEVELS, MAX_TERMS = 3, 8   # STRASSEN_MAX_LEVELS, STRASSEN_MAX_TERMS

STATUS = {
    0: "STRASSEN_OK", -1: "STRASSEN_ERR_DIM", -2: "STRASSEN_ERR_LD", -3: "STRASSEN_ERR_NULL",
    -4: "STRASSEN_ERR_LEVELS", -5: "STRASSEN_ERR_UNSUPPORTED", -6: "STRASSEN_ERR_CUDA",
    -7: "STRASSEN_ERR_TIMEOUT", -8: "STRASSEN_ERR_ALLOC", -9: "STRASSEN_ERR_ARG",
    -10: "STRASSEN_ERR_SCRATCH_LIMIT",
}


class StrassenError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({status})")


class strassen_problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("lda", ctypes.c_int64), ("ldb", ctypes.c_int64), ("ldc", ctypes.c_int64),
                ("levels", ctypes.c_int), ("variant", ctypes.c_int)]


_lib: Optional[ctypes.CDLL] = None

# (name, restype, argtypes) of every entry point declared in include/strassen.h
_I64, _P, _I, _IP = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)
SIGNATURES = {
    "strassen_gemm": (_I, [_I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _I, _I, _I, _P]),
    "classical_gemm": (_I, [_I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P]),
    "strassen_gemm_batched": (_I, [_I, ctypes.POINTER(strassen_problem), _I, _P]),
    "strassen_select": (_I, [_I64, _I64, _I64, _I, _IP, _IP, _IP]),
    "strassen_workspace_size": (_I64, [_I64, _I64, _I64, _I, _I, _I]),
    "strassen_status_string": (ctypes.c_char_p, [_I]),
    "strassen_plan_table": (_I, [_I, _I, _IP, _IP, _IP, _IP, _IP, _IP]),
    "strassen_dgemm": (_I, [_I, _I, _I64, _I64, _I64, ctypes.c_double, _P, _I64, _P, _I64, ctypes.c_double,
                            _P, _I64, _I, _I, _I, _P]),
    "strassen_dgemm_ex": (_I, [_I, _I, _I64, _I64, _I64, ctypes.c_double, _P, _I64, _P, _I64, ctypes.c_double,
                               _P, _I64, _I, _I, _I, ctypes.c_uint, _P]),
    "strassen_gemm_ab_noalloc": (_I, [_I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _I, _P]),
    "strassen_dsyrk": (_I, [_I, _I, _I64, _I64, ctypes.c_double, _P, _I64, ctypes.c_double, _P, _I64, _I,
                            ctypes.c_uint, _P]),
    "strassen_device_status": (_I, [_P]),
    "strassen_tune_record": (_I, [_I64, _I64, _I64, _I, _I, _I, _I]),
    "strassen_tune_clear": (_I, []),
    "strassen_model_seconds": (ctypes.c_double, [_I64, _I64, _I64, _I, _I]),
    "strassen_mlp_param_count": (_I, []),
    "strassen_mlp_forward": (_I, [_P, _P, _I, _P, _P]),
    "strassen_mlp_loss_grad": (_I, [_P, _P, _P, _P, _I, ctypes.c_float, _P, _P]),
    "strassen_mlp_adam": (_I, [_P, _P, _P, _P, _I, _I, ctypes.c_float, _P]),
    "strassen_selector_load": (_I, [ctypes.POINTER(ctypes.c_float), _I]),
    "strassen_selector_use": (_I, [_I, _I]),
    "strassen_selector_clear": (_I, []),
    "strassen_selector_candidate": (_I, [_I, _IP, _IP, _IP]),
    "strassen_selector_features": (_I, [_I64, _I64, _I64, _I, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint)]),
    "strassen_check_wait_timeout": (_I, [_I64, _P]),
    "strassen_profile_split_precision": (_I, [_I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _I,
                                              ctypes.POINTER(ctypes.c_float), _P]),
    "strassen_check_int_fadd": (_I, [_I64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), _P]),
}


def lib() -> ctypes.CDLL:
    """Load (building first if the sources changed) and return the CUDA library."""
    global _lib
    if _lib is None:
        from . import build as _build
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing: {path}")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, where: str) -> int:
    if status != 0:
        raise StrassenError(status, where)
    return status


# ---------------------------------------------------------------- raw entry points

def strassen_gemm(m, n, k, A, lda, B, ldb, C, ldc, levels, variant, dtype, stream) -> int:
    """C += A*B (device pointers as ints; stream as a cudaStream_t handle int)."""
    return lib().strassen_gemm(m, n, k, A, lda, B, ldb, C, ldc, levels, variant, dtype, stream)


def classical_gemm(m, n, k, A, lda, B, ldb, C, ldc, stream) -> int:
    return lib().classical_gemm(m, n, k, A, lda, B, ldb, C, ldc, stream)


def strassen_dgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, levels, variant, dtype,
                   stream) -> int:
    """C = alpha op(A) op(B) + beta C (row-major BLAS semantics); returns the status."""
    return lib().strassen_dgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, levels, variant,
                                dtype, stream)


def strassen_dgemm_ex(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, levels, variant, dtype,
                      flags, stream) -> int:
    """strassen_dgemm with flags (STRASSEN_FLAG_DETERMINISTIC); returns the status."""
    return lib().strassen_dgemm_ex(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, levels, variant,
                                   dtype, flags, stream)


def strassen_dsyrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, levels, flags, stream) -> int:
    """C = alpha op(A) op(A)^T + beta C on one triangle; returns the status."""
    return lib().strassen_dsyrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, levels, flags, stream)


def strassen_gemm_ab_noalloc(m, n, k, A, lda, B, ldb, C, ldc, levels, stream) -> int:
    """AB Strassen with its temporary in the library's fixed device array: no device
    allocation in the call (for callers that cannot allocate while they run)."""
    return lib().strassen_gemm_ab_noalloc(m, n, k, A, lda, B, ldb, C, ldc, levels, stream)


def strassen_gemm_batched(count, probs, dtype, stream) -> int:
    return lib().strassen_gemm_batched(count, probs, dtype, stream)


def strassen_device_status(stream) -> int:
    return lib().strassen_device_status(stream)


def strassen_check_wait_timeout(limit_cycles, stream) -> int:
    return lib().strassen_check_wait_timeout(limit_cycles, stream)


def strassen_check_int_fadd(count, seed, stream=0) -> int:
    """Number of hashed pairs where the library's integer-pipe addition differs from
    the hardware FP64 addition on this device (raises on error)."""
    mm = ctypes.c_uint64(0)
    _check(lib().strassen_check_int_fadd(count, seed, ctypes.byref(mm), stream), "strassen_check_int_fadd")
    return mm.value


def strassen_profile_split_precision(m, n, k, A, lda, B, ldb, C, ldc, levels, stream):
    """One split-precision product C += A*B with CUDA events between its stages;
    returns the milliseconds of (splits, slice products, recombination)."""
    ms = (ctypes.c_float * 3)()
    _check(lib().strassen_profile_split_precision(m, n, k, A, lda, B, ldb, C, ldc, levels, ms, stream),
           "strassen_profile_split_precision")
    return tuple(float(x) for x in ms)


def strassen_select(m, n, k, dtype):
    lv, var, tile = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    st = lib().strassen_select(m, n, k, dtype, ctypes.byref(lv), ctypes.byref(var), ctypes.byref(tile))
    _check(st, "strassen_select")
    return lv.value, var.value, tile.value


def strassen_tune_record(m, n, k, dtype, levels, variant, tile_id) -> int:
    return lib().strassen_tune_record(m, n, k, dtype, levels, variant, tile_id)


def strassen_tune_clear() -> int:
    return lib().strassen_tune_clear()


def strassen_model_seconds(m, n, k, levels, variant) -> float:
    return lib().strassen_model_seconds(m, n, k, levels, variant)


def strassen_mlp_param_count() -> int:
    return lib().strassen_mlp_param_count()


def strassen_mlp_forward(params, X, batch, Y, stream) -> int:
    return lib().strassen_mlp_forward(params, X, batch, Y, stream)


def strassen_mlp_loss_grad(params, X, T, mask, batch, mask_sum, grad, stream) -> int:
    return lib().strassen_mlp_loss_grad(params, X, T, mask, batch, mask_sum, grad, stream)


def strassen_mlp_adam(params, grad, m, v, count, step, lr, stream) -> int:
    return lib().strassen_mlp_adam(params, grad, m, v, count, step, lr, stream)


def strassen_selector_load(params_host, count) -> int:
    return lib().strassen_selector_load(params_host, count)


def strassen_selector_use(dtype, enable) -> int:
    return lib().strassen_selector_use(dtype, enable)


def strassen_selector_clear() -> int:
    return lib().strassen_selector_clear()


SELECTOR_CANDIDATES, SELECTOR_INPUTS = 16, 22  # STRASSEN_SELECTOR_CANDIDATES / _INPUTS


def strassen_selector_candidate(c):
    """(levels, variant, tile_id) of the learned selector's candidate c."""
    lv, var, tile = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().strassen_selector_candidate(c, ctypes.byref(lv), ctypes.byref(var), ctypes.byref(tile)),
           "strassen_selector_candidate")
    return lv.value, var.value, tile.value


def strassen_selector_features(m, n, k, dtype):
    """(x[22], base[16], valid mask) of a shape: the network's inputs, the analytic
    model's log2 seconds per candidate and the candidates valid for the dtype."""
    x = (ctypes.c_float * SELECTOR_INPUTS)()
    base = (ctypes.c_float * SELECTOR_CANDIDATES)()
    valid = ctypes.c_uint()
    _check(lib().strassen_selector_features(m, n, k, dtype, x, base, ctypes.byref(valid)),
           "strassen_selector_features")
    return list(x), list(base), valid.value


def strassen_workspace_size(m, n, k, levels, variant, dtype) -> int:
    return lib().strassen_workspace_size(m, n, k, levels, variant, dtype)


def strassen_status_string(status: int) -> str:
    return lib().strassen_status_string(status).decode()


def strassen_plan_table(levels: int):
    """The library's coefficient table for ``levels`` as a list of products, each a
    triple (a_terms, b_terms, c_terms) of (block_row, block_col, sign) tuples."""
    cap, w = 343, MAX_TERMS
    arrs = [(ctypes.c_int * cap)() for _ in range(3)] + [(ctypes.c_int * (w * cap))() for _ in range(3)]
    n = lib().strassen_plan_table(levels, cap, *arrs)
    if n < 0:
        raise StrassenError(n, "strassen_plan_table")
    na, nb, nc, ta, tb, tc = arrs

    def dec(v):
        return ((v // 2) // 16, (v // 2) % 16, -1 if v & 1 else 1)

    out = []
    for r in range(n):
        out.append((tuple(dec(ta[r * w + t]) for t in range(na[r])),
                    tuple(dec(tb[r * w + t]) for t in range(nb[r])),
                    tuple(dec(tc[r * w + t]) for t in range(nc[r]))))
    return out
