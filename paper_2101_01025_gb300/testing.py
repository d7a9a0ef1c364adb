"""Python side of include/aat_testing.h: single steps of the library for the
step-level parity tests, and host logic that needs no GPU."""
from __future__ import annotations

import ctypes

from ._native import PlanStats, check, lib


def is_prime(p: int) -> bool:
    return bool(lib().aatx_is_prime(p))


def sqrt_mod(a: int, p: int):
    r = lib().aatx_sqrt_mod(a, p)
    return None if r < 0 else int(r)


def sos(k: int, p: int):
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().aatx_sos(k, p, ctypes.byref(a), ctypes.byref(b)))
    return int(a.value), int(b.value)


def y_params(p: int):
    kind, a, b = ctypes.c_int(), ctypes.c_uint32(), ctypes.c_uint32()
    check(lib().aatx_y_params(p, ctypes.byref(kind), ctypes.byref(a), ctypes.byref(b)))
    return int(kind.value), int(a.value), int(b.value)


def digit_spec(p: int, with_sums: bool = False):
    """(b, L, dmax) of the digit split mod p; with_sums adds the number of
    pair-sum planes (0 when every digit pair is its own product)."""
    b, L, ns = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    dmax = (ctypes.c_int * 8)()
    check(lib().aatx_digit_spec(p, ctypes.byref(b), ctypes.byref(L), dmax, ctypes.byref(ns)))
    out = (int(b.value), int(L.value), [int(dmax[i]) for i in range(L.value)])
    return out + (int(ns.value),) if with_sums else out


def plan_stats(n: int, k: int, p: int, flags: int = 0) -> PlanStats:
    st = PlanStats()
    check(lib().aatx_plan_stats(n, k, p, flags, ctypes.byref(st)))
    return st


def leaf_groups(p: int, K: int, flags: int = 0, exact_bits: int = 0):
    """The leaf's group plan: (list of (xplane, yplane, kb0, kb1, kchunk, ratio),
    number of plane products)."""
    import numpy as np
    out = np.zeros((256, 6), dtype=np.int32)
    nprod = ctypes.c_int()
    ng = lib().aatx_leaf_groups(p, K, flags, exact_bits, out.ctypes.data, 256,
                                ctypes.byref(nprod))
    check(ng if ng < 0 else 0)
    return [tuple(int(v) for v in row) for row in out[:ng]], int(nprod.value)


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def sblocks(A, p: int):
    """S1..S4 of one level of Algorithm 1 (int32 CUDA tensors, canonical)."""
    import torch
    n, k = A.shape
    h, kap = n // 2, k // 2
    S = [torch.empty((h, kap), dtype=torch.int32, device=A.device) for _ in range(4)]
    check(lib().aatx_sblocks(A.data_ptr(), n, k, A.stride(0), p, *[s.data_ptr() for s in S],
                             kap, _stream()))
    return S


def split(X, p: int):
    """Digit planes of X as a (L, rows, kstride) bfloat16 CUDA tensor."""
    import torch
    rows, cols = X.shape
    _, L, _, ns = digit_spec(p, with_sums=True)
    ks = (cols + 7) // 8 * 8
    planes = torch.zeros((L + ns, rows, ks), dtype=torch.int16, device=X.device)
    check(lib().aatx_split(X.data_ptr(), rows, cols, X.stride(0), p, planes.data_ptr(),
                           _stream()))
    return planes.view(torch.bfloat16)


def leaf(X, Y, p: int, C=None, lower: bool = False, accumulate: bool = False,
         leafkind: int = 0, exact_bits: int = 0):
    """One leaf product C = X Y^T mod p (see aatx_leaf)."""
    import torch
    M, K = X.shape
    N = Y.shape[0]
    if C is None:
        C = torch.zeros((M, N), dtype=torch.int32, device=X.device)
    check(lib().aatx_leaf(X.data_ptr(), X.stride(0), Y.data_ptr(), Y.stride(0), M, N, K, p,
                          C.data_ptr(), C.stride(0), int(lower), int(accumulate), leafkind,
                          exact_bits, _stream()))
    return C


def postadd(C, h: int, p: int):
    check(lib().aatx_postadd(C.data_ptr(), C.stride(0), h, p, _stream()))
    return C
