"""Parity of the complex products with the FP64 oracle (GPU).

Error metric (per result): relative Frobenius error of the lower triangle,
||Low(C) - Low(C_ref)||_F / ||Low(C_ref)||_F, against the oracle's fp64
sums.  Bounds: 1e-5 for AAT_C_FP32 (3 BF16 pieces, 6 piece products),
1e-4 for AAT_C_BF16X3 (2 pieces: dropped terms of relative size 2^-16),
3e-3 for AAT_C_BF16 (plain BF16) in every form it is offered in: A A^H and
A A^T by 2M, and Algorithm 1 at depth 0; deeper Algorithm 1 is refused in
plain BF16.  Small-integer inputs are exact in every mode.
"""
import numpy as np
import pytest

import oracle
from paper_2101_01025_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1 << 16: 1e-4, 2 << 16: 3e-3}


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
    if flags == 2 << 16 and n * (n + 1) // 2 < 64:
        # a handful of entries: the Frobenius bound is a statement about many
        # rounding errors; one product of two BF16-rounded values can be off
        # by 2 * 2^-8 of |a||b|, so check that componentwise bound instead
        A64 = A.astype(np.complex128)
        mag = np.abs(A64.real) + np.abs(A64.imag)
        bound = 4 * 2.0**-8 * (mag @ mag.T) + 1e-6
        assert np.all(np.abs(np.tril(C) - np.tril(ref)) <= np.tril(bound))
    else:
        assert err <= TOL[flags], err
    if herm:
        d = np.diag(C)
        assert np.all(d.imag == 0) and np.all(d.real >= 0)
        # the diagonal is summed in FP64: close to the oracle's sums
        assert np.allclose(d.real, np.diag(ref).real, rtol=1e-6, atol=0)


@pytest.mark.parametrize("herm", [True, False])
@pytest.mark.parametrize("flags", [0, 1 << 16, 2 << 16])
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


@pytest.mark.parametrize("ill", [False, True])
def test_complex_full_size_sampled(lib, ill):
    """8192 x 8192 complex A (Re, Im i.i.d. N(0, 1), and the ill-scaled
    variant), A A^H and A A^T by 2M in every precision class: sampled
    entries at random positions and every 97th diagonal entry against the
    oracle, each class within its bound."""
    n = k = 8192
    A = synth.complex_normal(synth.SEED_BASE + 3 + (50 if ill else 0), (n, k), ill_scaled=ill)
    rng = np.random.default_rng(5)
    i = rng.integers(0, n, 3000)
    j = rng.integers(0, n, 3000)
    ij = np.stack([np.maximum(i, j), np.minimum(i, j)], 1)
    ij = np.concatenate([ij, np.array([[r, r] for r in range(0, n, 97)])])
    for herm in (True, False):
        ref = oracle.complex_entries(A.astype(np.complex128), ij, conj=herm)
        for flags in (0, 1 << 16, 2 << 16):
            C = run(lib, A, herm, flags)
            got = C[ij[:, 0], ij[:, 1]].astype(np.complex128)
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            print("2M n=k=8192 herm=%d ill=%d flags=%#x err=%.3e" % (herm, ill, flags, err))
            assert err <= TOL[flags], err


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

# Plain BF16 is offered at depth 0 only (where Algorithm 1 is the 2M form):
# each level forms sums and differences of blocks (S1..S4, U1..U5) whose BF16
# rounding is relative to the larger intermediate blocks, so the error grows
# past 3e-3 and those depths are refused.
TOL_ALG1 = {0: 1e-5, 1 << 16: 1e-4, 2 << 16: 3e-3}


@pytest.mark.parametrize("flags", [0, 1 << 16, 2 << 16])
@pytest.mark.parametrize("n,k", [(300, 200), (513, 640), (256, 512), (128, 64), (3, 5)])
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_aat_complex_alg1_matches_oracle(lib, flags, n, k, levels):
    A = synth.complex_normal(n * 3 + k + levels, (n, k))
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    if flags == 2 << 16 and levels > 0:
        with pytest.raises(lib.AatError) as ei:
            lib.aat_complex(Ad, flags=flags, levels=levels)
        assert ei.value.code == lib._native.AAT_EUNSUPPORTED
        return
    C = lib.aat_complex(Ad, flags=flags, levels=levels)
    torch.cuda.synchronize()
    ref = oracle.complex_low(A.astype(np.complex128), conj=False)
    err = rel_low_err(C.cpu().numpy(), ref)
    assert err <= TOL_ALG1[flags], err


def test_aat_complex_bf16_default_depth_is_zero(lib):
    """Without level bits, plain BF16 runs Algorithm 1 at depth 0 (the 2M
    form) even where the FP32 classes would recurse (n/2 >= 4096)."""
    n, k = 8192, 4096
    A = synth.complex_normal(synth.SEED_BASE + 41, (n, k))
    Ad = torch.from_numpy(A).cuda()
    C = lib.aat_complex(Ad, flags=2 << 16)
    torch.cuda.synchronize()
    ij = _sample_ij(n, 2000, 41)
    ref = oracle.complex_entries(A.astype(np.complex128), ij, conj=False)
    got = C[torch.from_numpy(ij[:, 0]).cuda(), torch.from_numpy(ij[:, 1]).cuda()]
    got = got.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 3e-3


def _sample_ij(n, count, seed):
    """Random lower entries, every block boundary of the recursion (rows and
    columns at multiples of n/4, +-1) and every 97th diagonal entry."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, n, count)
    j = rng.integers(0, n, count)
    ij = np.stack([np.maximum(i, j), np.minimum(i, j)], 1)
    edges = sorted({e + d for e in range(0, n + 1, n // 4) for d in (-1, 0) if 0 <= e + d < n})
    bd = np.array([[a, b] for a in edges for b in edges if a >= b])
    dg = np.array([[r, r] for r in range(0, n, 97)])
    return np.concatenate([ij, bd, dg])


@pytest.mark.parametrize("ill", [False, True])
def test_aat_complex_alg1_n8192_sampled(lib, ill):
    """Algorithm 1 over C (Y = i I) at n = k = 8192 (the complex workload),
    at 1 and 2 levels in the FP32 and 2-piece classes, plus plain BF16 at
    depth 0 (its only depth), on N(0, 1) entries and on the ill-scaled
    variant (row i times 10^u_i, u_i uniform in [-3, 3]): sampled entries
    against the oracle's FP64 sums, every class within its bound."""
    n = k = 8192
    A = synth.complex_normal(synth.SEED_BASE + 3 + (50 if ill else 0), (n, k), ill_scaled=ill)
    Ad = torch.from_numpy(A).cuda()
    ij = _sample_ij(n, 3000, 7)
    ref = oracle.complex_entries(A.astype(np.complex128), ij, conj=False)
    for flags, levels in [(0, 1), (0, 2), (1 << 16, 1), (1 << 16, 2), (2 << 16, 0)]:
        C = lib.aat_complex(Ad, flags=flags, levels=levels)
        torch.cuda.synchronize()
        got = C[torch.from_numpy(ij[:, 0]).cuda(), torch.from_numpy(ij[:, 1]).cuda()]
        got = got.cpu().numpy().astype(np.complex128)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print("Alg1 n=k=8192 ill=%d flags=%#x levels=%d err=%.3e" % (ill, flags, levels, err))
        assert err <= TOL_ALG1[flags], (flags, levels, err)
        del C
    with pytest.raises(lib.AatError):
        lib.aat_complex(Ad, flags=2 << 16, levels=1)


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
