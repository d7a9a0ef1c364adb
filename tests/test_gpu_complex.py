"""Parity of the complex products with the FP64 oracle (GPU).

Error metric (per result): relative Frobenius error of the lower triangle,
||Low(C) - Low(C_ref)||_F / ||Low(C_ref)||_F, against the oracle's fp64
sums.  Bounds: 1e-5 for AAT_C_FP32 (3 BF16 pieces, 6 piece products),
1e-4 for AAT_C_BF16X3 (2 pieces: dropped terms of relative size 2^-16),
3e-3 for AAT_C_BF16 with A A^H.  A A^T by 2M with plain BF16 gets 5e-3:
there Re C = G + H - H^T adds the BF16 rounding errors (2^-9 per input) of
three products of the same size as the result, and no FP64 diagonal takes
a large share of the norm.  Small-integer inputs are exact in every mode.
"""
import numpy as np
import pytest

import oracle
from paper_2101_01025_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1 << 16: 1e-4, 2 << 16: 3e-3}
TOL_T_BF16 = 5e-3   # A A^T by 2M, plain BF16


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_01025_gb300 import build
    build.build()
    import paper_2101_01025_gb300 as aat
    aat.aat_device_status(reset=True)
    yield aat
    assert aat.aat_device_status() == 0


def rel_low_err(C, ref):
    # only Low(C) is defined: the upper triangle may hold any bits
    d = np.tril(C).astype(np.complex128) - np.tril(ref)
    return np.linalg.norm(d) / max(np.linalg.norm(np.tril(ref)), 1e-300)


def run(lib, A, herm, flags):
    Ad = torch.from_numpy(np.ascontiguousarray(A.astype(np.complex64))).cuda()
    fn = lib.aah_complex if herm else lib.aat_complex_2m
    C = fn(Ad, flags=flags)
    torch.cuda.synchronize()
    return C.cpu().numpy()


@pytest.mark.parametrize("herm", [True, False])
@pytest.mark.parametrize("flags", [0, 1 << 16, 2 << 16])
@pytest.mark.parametrize("n,k", [(1, 1), (17, 33), (300, 200), (513, 640), (128, 64)])
def test_complex_matches_oracle(lib, herm, flags, n, k):
    A = synth.complex_normal(n * 7 + k, (n, k))
    C = run(lib, A, herm, flags)
    ref = oracle.complex_low(A.astype(np.complex128), conj=herm)
    err = rel_low_err(C, ref)
    tol = TOL_T_BF16 if (not herm and flags == 2 << 16) else TOL[flags]
    assert err <= tol, err
    if herm:
        d = np.diag(C)
        assert np.all(d.imag == 0) and np.all(d.real >= 0)
        # the diagonal is summed in FP64: close to the oracle's sums
        assert np.allclose(d.real, np.diag(ref).real, rtol=1e-6, atol=0)


@pytest.mark.parametrize("herm", [True, False])
@pytest.mark.parametrize("flags", [0, 1 << 16])
def test_complex_ill_scaled_rows(lib, herm, flags):
    A = synth.complex_normal(99, (400, 300), ill_scaled=True)
    C = run(lib, A, herm, flags)
    ref = oracle.complex_low(A.astype(np.complex128), conj=herm)
    assert rel_low_err(C, ref) <= TOL[flags]


@pytest.mark.parametrize("herm", [True, False])
@pytest.mark.parametrize("flags", [0, 1 << 16, 2 << 16])
def test_complex_small_integers_exact(lib, herm, flags):
    """Integers |x| <= 8 are exact in BF16 and every partial sum here is an
    integer below 2^24, so every mode is exact."""
    rng = np.random.default_rng(4)
    n, k = 260, 300
    A = rng.integers(-8, 9, (n, k)) + 1j * rng.integers(-8, 9, (n, k))
    C = run(lib, A, herm, flags)
    ref = oracle.complex_low(A.astype(np.complex128), conj=herm)
    assert np.array_equal(np.tril(C.astype(np.complex128)), np.tril(ref))


def test_complex_full_size_sampled(lib):
    """8192 x 8192 complex A (Re, Im i.i.d. N(0, 1)): sampled entries at
    every 32-row boundary and random positions against the oracle."""
    n = k = 8192
    A = synth.complex_normal(synth.SEED_BASE + 3, (n, k))
    for herm in (True, False):
        C = run(lib, A, herm, 0)
        rng = np.random.default_rng(5)
        i = rng.integers(0, n, 3000)
        j = rng.integers(0, n, 3000)
        ij = np.stack([np.maximum(i, j), np.minimum(i, j)], 1)
        ij = np.concatenate([ij, np.array([[r, r] for r in range(0, n, 97)])])
        ref = oracle.complex_entries(A.astype(np.complex128), ij, conj=herm)
        got = C[ij[:, 0], ij[:, 1]].astype(np.complex128)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-5, err


def test_complex_n16384_sampled(lib):
    """A A^H at n = k = 16384 (Re, Im i.i.d. N(0, 1), drawn on the device from a
    seeded generator), FP32 pieces: 3000 random lower entries and every 97th
    diagonal entry against the oracle's FP64 sums over the same rows."""
    n = k = 16384
    g = torch.Generator(device="cuda")
    g.manual_seed(synth.SEED_BASE + 4)
    Ad = torch.view_as_complex(torch.randn((n, k, 2), device="cuda", generator=g))
    C = lib.aah_complex(Ad, flags=0)
    torch.cuda.synchronize()
    rng = np.random.default_rng(6)
    i = rng.integers(0, n, 3000)
    j = rng.integers(0, n, 3000)
    ij = np.stack([np.maximum(i, j), np.minimum(i, j)], 1)
    ij = np.concatenate([ij, np.array([[r, r] for r in range(0, n, 97)])])
    rows = np.unique(ij)
    A_sub = Ad[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.complex128)
    ref = oracle.complex_entries(A_sub, np.searchsorted(rows, ij), conj=True)
    got = C[torch.from_numpy(ij[:, 0]).cuda(), torch.from_numpy(ij[:, 1]).cuda()]
    got = got.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err
    d = got[ij[:, 0] == ij[:, 1]]
    assert np.all(d.imag == 0) and np.all(d.real >= 0)
    assert np.allclose(d.real, ref[ij[:, 0] == ij[:, 1]].real, rtol=1e-6, atol=0)


# ----------------------------------------- A A^T over C by Algorithm 1 (Y = iI)

# Plain BF16 through the recursion: each level forms sums and differences
# of blocks (S1..S4, U1..U5) whose BF16 input rounding (2^-9) is relative to
# the larger intermediate blocks, so the error grows with the depth.
TOL_ALG1 = {0: 1e-5, 1 << 16: 1e-4}
TOL_ALG1_BF16 = {0: 5e-3, 1: 1e-2, 2: 4e-2}


@pytest.mark.parametrize("flags", [0, 1 << 16, 2 << 16])
@pytest.mark.parametrize("n,k", [(300, 200), (513, 640), (256, 512), (128, 64), (3, 5)])
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_aat_complex_alg1_matches_oracle(lib, flags, n, k, levels):
    A = synth.complex_normal(n * 3 + k + levels, (n, k))
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    C = lib.aat_complex(Ad, flags=flags, levels=levels)
    torch.cuda.synchronize()
    ref = oracle.complex_low(A.astype(np.complex128), conj=False)
    err = rel_low_err(C.cpu().numpy(), ref)
    tol = TOL_ALG1_BF16[levels] if flags == 2 << 16 else TOL_ALG1[flags]
    assert err <= tol, err


def test_aat_complex_alg1_small_integers_exact(lib):
    """Y = i I only swaps parts and flips a sign, so with small integers every
    intermediate value of the recursion is an exact integer."""
    rng = np.random.default_rng(12)
    n, k = 256, 192
    A = rng.integers(-4, 5, (n, k)) + 1j * rng.integers(-4, 5, (n, k))
    Ad = torch.from_numpy(A.astype(np.complex64)).cuda()
    for levels in (1, 2):
        C = lib.aat_complex(Ad, levels=levels)
        torch.cuda.synchronize()
        ref = oracle.complex_low(A.astype(np.complex128), conj=False)
        assert np.array_equal(np.tril(C.cpu().numpy().astype(np.complex128)), np.tril(ref))
