"""GB300 (sm_103a) library for the product of a matrix by its adjoint.

Python binding of the C ABI in ``include/aat.h``: the functions below carry
the C names and only marshal arguments (torch tensors -> device pointers,
the current torch stream -> cudaStream_t).  Every step runs in the CUDA
library ``libaat_gb300.so``; when it is missing the calls raise.

    aat_modp(A, p)            Low(A A^T) mod p, Algorithm 1 (Sec. 3)
    aat_gemm_modp(X, Y, p)    X Y^T mod p with the same exact leaf kernels
    aat_modp_host(A_np, p)    end to end from host memory
    aah_complex(A)            Low(A A^H) over C, Algorithm 2 (Sec. 6.1)
"""
from __future__ import annotations

import ctypes
import os

from . import _native
from ._native import (AAT_C_BF16, AAT_C_BF16X3, AAT_C_FP32, AAT_DIGITS_PLAIN,  # noqa: F401
                      AAT_IN_BALANCED, AAT_LEAF_F64, AAT_LEAF_I8, AAT_LEAF_SIMT, AAT_LEAF_TC,
                      AAT_LEVELS, AAT_LOW_MEMORY, AAT_WINOGRAD, AAT_ZERO_UPPER, AatError,
                      PlanStats, check, last_error, lib)

__all__ = [
    "aat_modp", "aat_syrk_modp", "aah_quat_modp", "aat_gemm_modp", "aat_modp_host", "aat_modp_host_d2h_bytes", "aat_workspace_size", "aat_set_workspace_limit",
    "aat_device_status", "tune_modp", "tune_lookup", "tune_save", "tune_load", "tune_clear",
    "aat_shutdown", "aat_version", "aah_complex", "aat_complex_2m", "aat_complex", "Plan", "AAT_LEVELS", "AAT_LEAF_TC", "AAT_LEAF_SIMT",
    "AAT_ZERO_UPPER", "AAT_IN_BALANCED", "AatError",
]


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _check_mat(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.int32 or t.dim() != 2:
        raise TypeError("%s must be a 2-D int32 tensor" % name)
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError("%s must have unit stride along rows" % name)
    return max(t.stride(0), t.shape[1], 1)


def aat_modp(A, p: int, C=None, flags: int = 0, levels: int | None = None, stream=None):
    """Low(A A^T) mod p into C (n x n int32, allocated if None); returns C.

    Only the lower triangle (diagonal included) of C is defined unless
    AAT_ZERO_UPPER is in ``flags``."""
    import torch
    lda = _check_mat(A, "A")
    n, k = A.shape
    if C is None:
        C = torch.empty((n, n), dtype=torch.int32, device=A.device)
    ldc = _check_mat(C, "C")
    if levels is not None:
        flags |= AAT_LEVELS(levels)
    check(lib().aat_modp_ex(A.data_ptr(), n, k, lda, p, C.data_ptr(), ldc, flags,
                            _stream(stream)))
    return C


def aat_gemm_modp(X, Y, p: int, C=None, flags: int = 0, stream=None):
    """X Y^T mod p (all entries) into C (allocated if None); returns C."""
    import torch
    ldx = _check_mat(X, "X")
    ldy = _check_mat(Y, "Y")
    m, k = X.shape
    n, k2 = Y.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.empty((m, n), dtype=torch.int32, device=X.device)
    ldc = _check_mat(C, "C")
    check(lib().aat_gemm_modp(X.data_ptr(), ldx, Y.data_ptr(), ldy, m, n, k, p, C.data_ptr(),
                              ldc, flags, _stream(stream)))
    return C


def aat_syrk_modp(alpha: int, A, beta: int, C, p: int, flags: int = 0,
                  levels: int | None = None, stream=None):
    """Low(C) <- alpha Low(A A^T) + beta Low(C) mod p in place (the SYRK
    form); C is an n x n int32 CUDA tensor holding residues |x| < p in its
    lower triangle; its strict upper triangle is used as scratch.  Returns C."""
    if levels is not None:
        flags |= AAT_LEVELS(levels)
    lda = _check_mat(A, "A")
    ldc = _check_mat(C, "C")
    n, k = A.shape
    if tuple(C.shape) != (n, n):
        raise ValueError("C must be n x n")
    check(lib().aat_syrk_modp(alpha % 2**32, A.data_ptr(), n, k, lda, beta % 2**32,
                              C.data_ptr(), ldc, p, flags, _stream(stream)))
    return C


def aah_quat_modp(A, B, C, D, p: int, H=None, flags: int = 0, levels: int | None = None,
                  stream=None):
    """Quaternion M M^H mod p for M = A + B i + C j + D k (four n x k int32
    CUDA tensors with the same row stride): returns (H1, H2, H3, H4), n x n
    int32 CUDA tensors holding Low of each part (H may pass four of them)."""
    import torch
    if levels is not None:
        flags |= AAT_LEVELS(levels)
    lda = _check_mat(A, "A")
    n, k = A.shape
    for X, nm in ((B, "B"), (C, "C"), (D, "D")):
        if _check_mat(X, nm) != lda or tuple(X.shape) != (n, k):
            raise ValueError("A, B, C, D must have the same shape and row stride")
    if H is None:
        H = tuple(torch.empty((n, n), dtype=torch.int32, device=A.device) for _ in range(4))
    ldh = _check_mat(H[0], "H1")
    for X in H[1:]:
        if _check_mat(X, "H") != ldh or tuple(X.shape) != (n, n):
            raise ValueError("H1..H4 must be n x n with the same row stride")
    check(lib().aah_quat_modp(A.data_ptr(), B.data_ptr(), C.data_ptr(), D.data_ptr(), n, k, lda,
                              p, H[0].data_ptr(), H[1].data_ptr(), H[2].data_ptr(),
                              H[3].data_ptr(), ldh, flags, _stream(stream)))
    return tuple(H)


def aat_modp_host(A, p: int, C=None, flags: int = 0, levels: int | None = None):
    """End to end from host memory: A is a C-contiguous int32 numpy array (or
    pinned CPU tensor); returns C (n x n, host, same kind as A).  Only the
    lower triangle of C is written unless AAT_ZERO_UPPER is set."""
    import numpy as np
    if levels is not None:
        flags |= AAT_LEVELS(levels)
    if isinstance(A, np.ndarray):
        A = np.ascontiguousarray(A, dtype=np.int32)
        n, k = A.shape
        if C is None:
            C = np.empty((n, n), dtype=np.int32)
        check(lib().aat_modp_host(A.ctypes.data, n, k, p, C.ctypes.data, flags))
        return C
    import torch
    if A.is_cuda or A.dtype != torch.int32 or not A.is_contiguous():
        raise TypeError("A must be a contiguous int32 host tensor")
    n, k = A.shape
    if C is None:
        C = torch.empty((n, n), dtype=torch.int32, pin_memory=A.is_pinned())
    check(lib().aat_modp_host(A.data_ptr(), n, k, p, C.data_ptr(), flags))
    return C


def tune_modp(n: int, k: int, p: int, flags: int = 0, reps: int = 3, stream=None) -> dict:
    """Autotune Low(A A^T) mod p for shape (n, k): recursion levels, leaf
    kernel form and digit-product form, timed on synthetic residues on the
    GPU; the choice is kept for later calls of that shape and returned."""
    from ._native import Tune
    t = Tune()
    check(lib().aat_tune_modp(n, k, p, flags, reps, _stream(stream), ctypes.byref(t)))
    return t.as_dict()


def tune_lookup(n: int, k: int, p: int):
    """The tuned choice for (n, k, p), or None."""
    from ._native import Tune
    t = Tune()
    return t.as_dict() if lib().aat_tune_lookup(n, k, p, ctypes.byref(t)) else None


def tune_save(path: str) -> int:
    r = lib().aat_tune_save(os.fsencode(path))
    check(min(r, 0))
    return r


def tune_load(path: str) -> int:
    r = lib().aat_tune_load(os.fsencode(path))
    check(min(r, 0))
    return r


def tune_clear() -> None:
    lib().aat_tune_clear()


def aat_modp_host_d2h_bytes(n: int, flags: int = 0) -> int:
    """Bytes aat_modp_host copies back to the host for an n x n result."""
    return int(lib().aat_modp_host_d2h_bytes(n, flags))


def _check_cmat(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.complex64 or t.dim() != 2:
        raise TypeError("%s must be a 2-D complex64 tensor" % name)
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError("%s must have unit stride along rows" % name)
    return max(t.stride(0), t.shape[1], 1)


def aah_complex(A, C=None, flags: int = 0, stream=None):
    """Low(A A^H) for a complex64 CUDA matrix A by Algorithm 2 (2M); returns C.

    flags: AAT_C_FP32 (default), AAT_C_BF16X3 or AAT_C_BF16."""
    import torch
    lda = _check_cmat(A, "A")
    n, k = A.shape
    if C is None:
        C = torch.empty((n, n), dtype=torch.complex64, device=A.device)
    ldc = _check_cmat(C, "C")
    check(lib().aah_complex_ex(A.data_ptr(), n, k, lda, C.data_ptr(), ldc, flags,
                               _stream(stream)))
    return C


def aat_complex_2m(A, C=None, flags: int = 0, stream=None):
    """Low(A A^T) for a complex64 CUDA matrix A by Algorithm 2 with eps = -1."""
    import torch
    lda = _check_cmat(A, "A")
    n, k = A.shape
    if C is None:
        C = torch.empty((n, n), dtype=torch.complex64, device=A.device)
    ldc = _check_cmat(C, "C")
    check(lib().aat_complex_2m(A.data_ptr(), n, k, lda, C.data_ptr(), ldc, flags,
                               _stream(stream)))
    return C


def aat_complex(A, C=None, flags: int = 0, levels: int | None = None, stream=None):
    """Low(A A^T) for a complex64 CUDA matrix A by Algorithm 1 with Y = i I."""
    import torch
    lda = _check_cmat(A, "A")
    n, k = A.shape
    if C is None:
        C = torch.empty((n, n), dtype=torch.complex64, device=A.device)
    ldc = _check_cmat(C, "C")
    if levels is not None:
        flags |= AAT_LEVELS(levels)
    check(lib().aat_complex_ex(A.data_ptr(), n, k, lda, C.data_ptr(), ldc, flags,
                               _stream(stream)))
    return C


class Plan:
    """A batch of independent products executed as one CUDA graph launch.

    problems: list of (kind, A, C, p, flags) with kind "modp" (int32 CUDA
    tensors, field p), "aah" or "aat_c" (complex64 CUDA tensors).  The
    tensors must stay alive and keep their storage while the plan lives."""

    KINDS = {"modp": _native.AAT_KIND_MODP, "aah": _native.AAT_KIND_AAH,
             "aat_c": _native.AAT_KIND_AAT_C}

    def __init__(self, problems):
        import ctypes
        arr = (_native.Problem * len(problems))()
        self._keep = []
        for i, (kind, A, C, p, flags) in enumerate(problems):
            chk = _check_mat if kind == "modp" else _check_cmat
            lda = chk(A, "A")
            ldc = chk(C, "C")
            arr[i] = _native.Problem(self.KINDS[kind], A.data_ptr(), C.data_ptr(), A.shape[0],
                                     A.shape[1], lda, ldc, p or 0, flags)
            self._keep += [A, C]
        h = ctypes.c_void_p()
        check(lib().aat_plan_create(arr, len(problems), ctypes.byref(h)))
        self._h = h

    def execute(self, stream=None):
        check(lib().aat_plan_execute(self._h, _stream(stream)))

    def info(self):
        import ctypes
        b, s, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        check(lib().aat_plan_info(self._h, ctypes.byref(b), ctypes.byref(s), ctypes.byref(w)))
        return {"batched": b.value, "solo": s.value, "workspace": w.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().aat_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def aat_workspace_size(n: int, k: int, p: int, flags: int = 0) -> int:
    return int(lib().aat_workspace_size(n, k, p, flags))


def aat_set_workspace_limit(nbytes: int | None) -> None:
    """Products whose fast schedule needs more workspace than ``nbytes`` run
    the low-memory schedule (AAT_LOW_MEMORY); None removes the limit."""
    lib().aat_set_workspace_limit(2**64 - 1 if nbytes is None else int(nbytes))


def aat_device_status(reset: bool = False) -> int:
    return int(lib().aat_device_status(1 if reset else 0))


def aat_shutdown() -> None:
    lib().aat_shutdown()


def aat_version() -> int:
    return int(lib().aat_version())
