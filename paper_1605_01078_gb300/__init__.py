"""Strassen's algorithm fused into GEMM on GB300 (sm_103a).

Implements the family of Huang, Smith, Henry and van de Geijn, "Implementing
Strassen's Algorithm with BLIS" (arXiv:1605.01078): one-, two- and three-level Strassen in the
ABC, AB and Naive variants plus the classical product, behind the C ABI of
``include/strassen.h``.  This package is the thin Python side of that ABI:

* :mod:`._binding` -- the C entry points under the same names (ctypes marshalling);
* :func:`gemm`, :func:`classical` -- the same calls taking torch CUDA tensors, which
  supply device memory and the stream only.

All arithmetic runs in the library's CUDA kernels; a missing library is an error.
"""
from __future__ import annotations

from . import _binding
from ._binding import (STRASSEN_AB, STRASSEN_ABC, STRASSEN_AUTO, STRASSEN_F64, STRASSEN_HYBRID,  # noqa: F401
                       STRASSEN_F64_OZ_BF16, STRASSEN_F64_OZ_INT8, STRASSEN_FLAG_DETERMINISTIC, STRASSEN_NAIVE,
                       StrassenError,
                       classical_gemm, strassen_gemm, strassen_gemm_ab_noalloc, strassen_gemm_batched,
                       strassen_dgemm, strassen_dgemm_ex, strassen_dsyrk,
                       strassen_plan_table,
                       strassen_problem, strassen_select, strassen_status_string, strassen_device_status,
                       strassen_check_wait_timeout, strassen_tune_record, strassen_tune_clear,
                       strassen_model_seconds, strassen_mlp_param_count, strassen_mlp_forward,
                       strassen_mlp_loss_grad, strassen_mlp_adam, strassen_selector_load,
                       strassen_selector_clear, strassen_check_int_fadd, strassen_selector_use,
                       strassen_workspace_size, strassen_profile_split_precision,
                       strassen_selector_candidate, strassen_selector_features)

VARIANTS = {"ABC": STRASSEN_ABC, "AB": STRASSEN_AB, "NAIVE": STRASSEN_NAIVE, "AUTO": STRASSEN_AUTO,
            "HYBRID": STRASSEN_HYBRID}
DTYPES = {"f64": STRASSEN_F64, "oz_int8": STRASSEN_F64_OZ_INT8, "oz_bf16": STRASSEN_F64_OZ_BF16}


def _mat(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.dim() != 2:
        raise TypeError(f"{name} must be a 2-D torch.float64 tensor")
    if not t.is_cuda:
        raise TypeError(f"{name} must live on a CUDA device")
    if t.stride(1) != 1 and t.size(1) > 1:
        raise TypeError(f"{name} must be row-major with unit column stride")
    return t


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ld(t):
    return max(t.stride(0), t.size(1), 1)


def gemm(A, B, C, levels: int = 1, variant="ABC", dtype="f64", stream=None, deterministic: bool = False) -> None:
    """In place on the stream: C += A @ B with ``levels`` levels of Strassen.  With
    ``deterministic`` the call goes through strassen_dgemm_ex with
    STRASSEN_FLAG_DETERMINISTIC (fixed rounding order)."""
    A, B, C = _mat(A, "A"), _mat(B, "B"), _mat(C, "C")
    m, k = A.shape
    k2, n = B.shape
    if k2 != k or tuple(C.shape) != (m, n):
        raise ValueError(f"shape mismatch: A {tuple(A.shape)}, B {tuple(B.shape)}, C {tuple(C.shape)}")
    v = VARIANTS[variant.upper()] if isinstance(variant, str) else int(variant)
    d = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    if deterministic:
        st = strassen_dgemm_ex(0, 0, m, n, k, 1.0, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), 1.0, C.data_ptr(),
                               _ld(C), int(levels), v, d, STRASSEN_FLAG_DETERMINISTIC, _stream(stream))
        _binding._check(st, "strassen_dgemm_ex")
        return
    st = strassen_gemm(m, n, k, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), C.data_ptr(), _ld(C),
                       int(levels), v, d, _stream(stream))
    _binding._check(st, "strassen_gemm")


def dgemm(A, B, C, alpha: float = 1.0, beta: float = 1.0, trans_a: bool = False, trans_b: bool = False,
          levels: int = 1, variant="ABC", dtype="f64", stream=None) -> None:
    """In place on the stream: C = alpha op(A) op(B) + beta C, op(X) = X.T when trans_x.
    A and B are the stored matrices (A is k x m when trans_a); transposes are read in
    place by the kernels."""
    A, B, C = _mat(A, "A"), _mat(B, "B"), _mat(C, "C")
    m, k = (A.shape[1], A.shape[0]) if trans_a else (A.shape[0], A.shape[1])
    k2, n = (B.shape[1], B.shape[0]) if trans_b else (B.shape[0], B.shape[1])
    if k2 != k or tuple(C.shape) != (m, n):
        raise ValueError(f"shape mismatch: op(A) {m}x{k}, op(B) {k2}x{n}, C {tuple(C.shape)}")
    v = VARIANTS[variant.upper()] if isinstance(variant, str) else int(variant)
    d = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    st = strassen_dgemm(int(bool(trans_a)), int(bool(trans_b)), m, n, k, float(alpha), A.data_ptr(), _ld(A),
                        B.data_ptr(), _ld(B), float(beta), C.data_ptr(), _ld(C), int(levels), v, d, _stream(stream))
    _binding._check(st, "strassen_dgemm")


def dsyrk(A, C, alpha: float = 1.0, beta: float = 1.0, lower: bool = True, trans: bool = False, levels: int = -1,
          deterministic: bool = False, stream=None) -> None:
    """In place on the stream: one triangle of C becomes alpha op(A) op(A)^T + beta C,
    op(A) = A.T when trans (A stored k x n)."""
    A, C = _mat(A, "A"), _mat(C, "C")
    n, k = (A.shape[1], A.shape[0]) if trans else (A.shape[0], A.shape[1])
    if tuple(C.shape) != (n, n):
        raise ValueError(f"shape mismatch: op(A) {n}x{k}, C {tuple(C.shape)}")
    st = strassen_dsyrk(0 if lower else 1, int(bool(trans)), n, k, float(alpha), A.data_ptr(), _ld(A), float(beta),
                        C.data_ptr(), _ld(C), int(levels), STRASSEN_FLAG_DETERMINISTIC if deterministic else 0,
                        _stream(stream))
    _binding._check(st, "strassen_dsyrk")


def classical(A, B, C, stream=None) -> None:
    """In place on the stream: C += A @ B by the library's classical FP64 kernel."""
    A, B, C = _mat(A, "A"), _mat(B, "B"), _mat(C, "C")
    m, k = A.shape
    k2, n = B.shape
    if k2 != k or tuple(C.shape) != (m, n):
        raise ValueError("shape mismatch")
    st = classical_gemm(m, n, k, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), C.data_ptr(), _ld(C),
                        _stream(stream))
    _binding._check(st, "classical_gemm")


def load_library():
    """Load the CUDA library (building it if needed) and return the ctypes handle."""
    return _binding.lib()
