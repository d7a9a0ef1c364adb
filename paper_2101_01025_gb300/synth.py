"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method: it only draws numbers.  It is
the one module both sides of a parity test may use.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), element t of a stream with seed s being
mix(s + (t + 1) * 0x9E3779B97F4A7C15) with the published finaliser.
Maps:
  * residue in [0, p): (z >> 32) * p >> 32   (multiply-shift; bias < p / 2^32)
  * uniform in (0, 1): ((z >> 11) + 0.5) / 2^53
  * standard normal: Box-Muller on two consecutive uniforms.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: Seed base of the workloads (seed = base + workload index).
SEED_BASE = 0x2101010250


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` consecutive SplitMix64 outputs (uint64) of stream ``seed``."""
    with np.errstate(over="ignore"):
        t = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + t * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def residues(seed: int, shape, p: int, balanced: bool = False,
             chunk: int = 1 << 24) -> np.ndarray:
    """int32 matrix of residues mod p, uniform in [0, p).

    With ``balanced`` the same draws are stored in (-p/2, p/2]: values above
    p // 2 are shifted down by p."""
    shape = tuple(int(s) for s in shape)
    count = int(np.prod(shape)) if shape else 1
    out = np.empty(count, dtype=np.int32)
    pp = np.uint64(p)
    for start in range(0, count, chunk):
        m = min(chunk, count - start)
        z = splitmix64(seed, m, offset=start)
        with np.errstate(over="ignore"):
            r = ((z >> np.uint64(32)) * pp) >> np.uint64(32)
        r = r.astype(np.int64)
        if balanced:
            r = np.where(r > p // 2, r - p, r)
        out[start:start + m] = r.astype(np.int32)
    return out.reshape(shape)


def uniforms(seed: int, count: int, offset: int = 0) -> np.ndarray:
    z = splitmix64(seed, count, offset)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) / float(1 << 53)


def complex_normal(seed: int, shape, ill_scaled: bool = False) -> np.ndarray:
    """complex64 matrix with Re, Im i.i.d. N(0, 1) (Box-Muller).

    ``ill_scaled``: row i is multiplied by 10**u_i, u_i uniform in (-3, 3)
    (drawn from stream seed + 1), so row norms spread over 1e-3 .. 1e3."""
    shape = tuple(int(s) for s in shape)
    count = int(np.prod(shape))
    u = uniforms(seed, 2 * count)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    re = rad * np.cos(2.0 * np.pi * u2)
    im = rad * np.sin(2.0 * np.pi * u2)
    A = (re + 1j * im).reshape(shape)
    if ill_scaled:
        e = uniforms(seed + 1, shape[0]) * 6.0 - 3.0
        A = A * (10.0 ** e)[:, None]
    return A.astype(np.complex64)


def log_uniform_ints(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers log-uniform in [lo, hi]."""
    u = uniforms(seed, count)
    v = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    return np.clip(np.floor(v).astype(np.int64), lo, hi)


def vectors_mod_p(seed: int, count: int, n: int, p: int) -> np.ndarray:
    """``count`` random vectors of length n over [0, p) (Freivalds checks)."""
    return residues(seed, (count, n), p).astype(np.uint32)
