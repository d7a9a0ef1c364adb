"""CPU oracle for Low(A A^T) mod p and for A A^H / A A^T over C.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The library
(``paper_2101_01025_gb300``) never imports it, and it never imports the
library: the two share no code.

Contents
--------
* ``aat_oracle.c`` -- the plain definitions in C (triple loops, exact
  ``unsigned __int128`` sums mod p, fp64 complex sums), Euler's criterion,
  Tonelli-Shanks, Algorithm 3 (SoS), the S blocks of Algorithm 1 and a
  Freivalds checker.  Built with gcc on first use (``build()``).
* ``alg1.py`` -- Algorithm 1 and Algorithm 2 restated step by step in the
  paper's order and notation on exact Python integers (small sizes only),
  used to pin the readings of the paper and the intermediate blocks.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, brute force, invariants, independent library routines).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aat_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP) into oracle/_build/liborc.so."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, u32, i32, u64 = ctypes.c_int64, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint64
        vp = ctypes.c_void_p
        lib.orc_num_threads.restype = i32
        lib.orc_aat_modp_low.argtypes = [vp, i64, i64, i64, u32, vp, i64, i32]
        lib.orc_aat_modp_entries.argtypes = [vp, i64, i64, i64, u32, vp, i64, vp, i32]
        lib.orc_gemm_modp.argtypes = [vp, i64, vp, i64, i64, i64, i64, u32, vp, i64, i32]
        lib.orc_freivalds_modp.argtypes = [vp, i64, i64, i64, vp, i64, u32, vp, i32, i32]
        lib.orc_complex_low.argtypes = [vp, i64, i64, i64, i32, vp, i64, i32]
        lib.orc_complex_entries.argtypes = [vp, i64, i64, i64, i32, vp, i64, vp, i32]
        lib.orc_is_prime.argtypes = [u64]
        lib.orc_legendre.argtypes = [i64, u64]
        lib.orc_sqrt_mod.argtypes = [i64, u64, ctypes.POINTER(u64)]
        lib.orc_sos_modp.argtypes = [i64, u64, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        lib.orc_build_y.argtypes = [i32, u32, u32, u32, i64, vp]
        lib.orc_alg1_sblocks.argtypes = [vp, i64, i64, i64, u32, i32, u32, u32, vp, vp, vp, vp]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i32(A) -> np.ndarray:
    A = np.ascontiguousarray(A)
    if A.dtype != np.int32:
        raise TypeError("expected an int32 array, got %s" % A.dtype)
    return A


def num_threads() -> int:
    return int(_load().orc_num_threads())


# ------------------------------------------------------------------ F_p

def aat_modp_low(A, p: int, threads: int = 0) -> np.ndarray:
    """Low(A A^T) mod p as an n x n uint32 array (strict upper part zero)."""
    A = _i32(A)
    n, k = A.shape
    C = np.zeros((n, n), dtype=np.uint32)
    rc = _load().orc_aat_modp_low(_ptr(A), n, k, k, p, _ptr(C), n, threads)
    if rc:
        raise ValueError("orc_aat_modp_low failed (%d)" % rc)
    return C


def syrk_modp_low(alpha: int, A, beta: int, C, p: int, threads: int = 0) -> np.ndarray:
    """Low(alpha A A^T + beta C) mod p, canonical, strict upper part zero:
    the SYRK update C <- alpha A A^T + beta C restricted to the lower
    triangle (Sec. 7, Table 4), written out from its definition: the exact
    product Low(A A^T) mod p, then each lower entry combined in exact
    integer arithmetic.  C may hold any residues (its upper part is ignored)."""
    P = aat_modp_low(A, p, threads).astype(np.int64)
    Cl = np.tril(np.asarray(C, dtype=np.int64) % p)
    out = ((alpha % p) * P + (beta % p) * Cl) % p
    return np.tril(out).astype(np.uint32)


def quat_aah_modp_low(A, B, C, D, p: int, threads: int = 0):
    """M M^H mod p for the quaternion matrix M = A + B i + C j + D k (n x k
    over F_p, i^2 = j^2 = k^2 = ijk = -1), M^H the conjugate transpose
    (Sec. 6.2): returns Low(H1), Low(H2), Low(H3), Low(H4) of
    H = H1 + H2 i + H3 j + H4 k as n x n uint32 arrays.  Written out from the
    definition: H[r, c] = sum_l M[r, l] conj(M[c, l]) with the Hamilton
    product (a1 + b1 i + c1 j + d1 k)(a2 - b2 i - c2 j - d2 k) =
        (a1 a2 + b1 b2 + c1 c2 + d1 d2)
      + (-a1 b2 + b1 a2 - c1 d2 + d1 c2) i
      + (-a1 c2 + b1 d2 + c1 a2 - d1 b2) j
      + (-a1 d2 - b1 c2 + c1 b2 + d1 a2) k,
    each sum of products over l one exact product X Y^T mod p (gemm_modp)."""
    Ms = [_i32(X) for X in (A, B, C, D)]
    prod = {}

    def g(x, y):
        if (x, y) not in prod:
            prod[(x, y)] = gemm_modp(Ms[x], Ms[y], p, threads).astype(np.int64)
        return prod[(x, y)]

    # (sign, index of the left factor's part, index of the right one's)
    terms = [
        [(1, 0, 0), (1, 1, 1), (1, 2, 2), (1, 3, 3)],
        [(-1, 0, 1), (1, 1, 0), (-1, 2, 3), (1, 3, 2)],
        [(-1, 0, 2), (1, 1, 3), (1, 2, 0), (-1, 3, 1)],
        [(-1, 0, 3), (-1, 1, 2), (1, 2, 1), (1, 3, 0)],
    ]
    out = []
    for comp in terms:
        H = sum(s * g(x, y) for s, x, y in comp) % p
        out.append(np.tril(H).astype(np.uint32))
    return tuple(out)


def aat_modp_entries(A, p: int, ij, threads: int = 0) -> np.ndarray:
    """(A A^T)[i, j] mod p at the given (i, j) pairs (array of shape (t, 2))."""
    A = _i32(A)
    n, k = A.shape
    ij = np.ascontiguousarray(np.asarray(ij, dtype=np.int64).reshape(-1, 2))
    out = np.zeros(ij.shape[0], dtype=np.uint32)
    rc = _load().orc_aat_modp_entries(_ptr(A), n, k, k, p, _ptr(ij), ij.shape[0],
                                      _ptr(out), threads)
    if rc:
        raise ValueError("orc_aat_modp_entries failed (%d)" % rc)
    return out


def gemm_modp(X, Y, p: int, threads: int = 0) -> np.ndarray:
    """X Y^T mod p (all entries), uint32."""
    X, Y = _i32(X), _i32(Y)
    m, k = X.shape
    n, k2 = Y.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    C = np.zeros((m, n), dtype=np.uint32)
    _load().orc_gemm_modp(_ptr(X), k, _ptr(Y), k, m, n, k, p, _ptr(C), n, threads)
    return C


def freivalds_modp(A, C, p: int, xs, threads: int = 0) -> int:
    """Number of vectors x (rows of ``xs``) for which Sym(C) x != A (A^T x)."""
    A = _i32(A)
    C = _i32(C)
    n, k = A.shape
    xs = np.ascontiguousarray(np.asarray(xs, dtype=np.uint32).reshape(-1, n))
    return int(_load().orc_freivalds_modp(_ptr(A), n, k, k, _ptr(C), C.shape[1], p,
                                          _ptr(xs), xs.shape[0], threads))


# ------------------------------------------------------------------ C

def _c128(A) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(A, dtype=np.complex128))


def complex_low(A, conj: bool = True, threads: int = 0) -> np.ndarray:
    """Low(A A^H) (conj=True) or Low(A A^T) (conj=False) in fp64, complex128."""
    A = _c128(A)
    n, k = A.shape
    C = np.zeros((n, n), dtype=np.complex128)
    _load().orc_complex_low(_ptr(A), n, k, k, 1 if conj else 0, _ptr(C), n, threads)
    return C


def complex_entries(A, ij, conj: bool = True, threads: int = 0) -> np.ndarray:
    A = _c128(A)
    n, k = A.shape
    ij = np.ascontiguousarray(np.asarray(ij, dtype=np.int64).reshape(-1, 2))
    out = np.zeros(ij.shape[0], dtype=np.complex128)
    _load().orc_complex_entries(_ptr(A), n, k, k, 1 if conj else 0, _ptr(ij),
                                ij.shape[0], _ptr(out), threads)
    return out


# ------------------------------------------------------------ number theory

def is_prime(p: int) -> bool:
    return bool(_load().orc_is_prime(p))


def legendre(a: int, p: int) -> int:
    return int(_load().orc_legendre(a, p))


def sqrt_mod(a: int, p: int):
    """Square root of a mod p (the smaller of +-r), or None for a non-square."""
    r = ctypes.c_uint64(0)
    ok = _load().orc_sqrt_mod(a, p, ctypes.byref(r))
    return int(r.value) if ok else None


def sos_modp(k: int, p: int):
    """Algorithm 3: (a, b) with a^2 + b^2 == k (mod p)."""
    a, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
    ok = _load().orc_sos_modp(k, p, ctypes.byref(a), ctypes.byref(b))
    if not ok:
        raise ValueError("SoS failed for p=%d" % p)
    return int(a.value), int(b.value)


def skew_unitary_params(p: int):
    """(ykind, ya, yb) of a skew-unitary Y for the transposition over F_p.

    p == 1 mod 4: Y = i I with i^2 == -1 (Sec. 4.2), ykind 1.
    p == 3 mod 4: Y = [[a, b], [-b, a]] (x) I with a^2 + b^2 == -1 found by
    Algorithm 3 (Sec. 4.3), ykind 2.
    """
    if p % 4 == 1:
        r = sqrt_mod(p - 1, p)
        return 1, r, 0
    a, b = sos_modp(-1, p)
    return 2, a, b


def build_y(ykind: int, ya: int, yb: int, p: int, kappa: int) -> np.ndarray:
    Y = np.zeros((kappa, kappa), dtype=np.uint32)
    rc = _load().orc_build_y(ykind, ya, yb, p, kappa, _ptr(Y))
    if rc:
        raise ValueError("bad Y parameters")
    return Y


def alg1_sblocks(A, p: int, ykind: int, ya: int, yb: int):
    """S1, S2, S3, S4 of Algorithm 1 (canonical, uint32), each n/2 x k/2."""
    A = _i32(A)
    n, k = A.shape
    h, kap = n // 2, k // 2
    outs = [np.zeros((h, kap), dtype=np.uint32) for _ in range(4)]
    rc = _load().orc_alg1_sblocks(_ptr(A), n, k, k, p, ykind, ya, yb,
                                  *[_ptr(o) for o in outs])
    if rc:
        raise ValueError("orc_alg1_sblocks failed (%d)" % rc)
    return tuple(outs)
