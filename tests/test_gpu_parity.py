"""Parity of the CUDA path with the CPU oracle (run on a GB300 with -m gpu).

Every comparison over F_p is bit-exact.  Small cases span several 128 x 256
output tiles with ragged tails; full-size cases compare sampled entries (at
every recursion block boundary) one by one with the oracle and check the
whole result with Freivalds' test.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_2101_01025_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRIMES = [65521, 131071, 2**31 - 1]


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_01025_gb300 import build
    build.build()
    import paper_2101_01025_gb300 as aat
    aat.aat_device_status(reset=True)
    yield aat
    assert aat.aat_device_status() == 0, "a bounded device wait gave up"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def bal(x, p):
    x = np.asarray(x, dtype=np.int64) % p
    return np.where(x > (p - 1) // 2, x - p, x)


def low_equal(C, ref):
    C = np.asarray(C, dtype=np.int64)
    ref = np.asarray(ref, dtype=np.int64)
    return np.array_equal(np.tril(C), np.tril(ref))


# ------------------------------------------------------------ single steps

@pytest.mark.parametrize("p", PRIMES + [13])
def test_split_reconstructs_balanced_residues(p):
    from paper_2101_01025_gb300 import testing as T
    b, L, dmax, ns = T.digit_spec(p, with_sums=True)
    half = (p - 1) // 2
    X = synth.residues(1, (37, 203), p, balanced=True)
    X[0, :7] = [half, -half, 0, 1, -1, half - 1, -(half - 1)]
    X[1, :] = p - 1            # canonical input: the kernel balances it
    planes = T.split(dev(X), p).float().cpu().numpy()[:, :, :203]
    assert planes.shape[0] == L + ns
    for d in range(L):
        assert np.all(np.abs(planes[d]) <= dmax[d])
        assert np.all(planes[d] == np.round(planes[d]))
    rec = sum(planes[d].astype(np.int64) << (b * d) for d in range(L))
    assert np.array_equal(rec, bal(X, p))
    pairs = [(i, j) for i in range(L) for j in range(i + 1, L)]
    assert ns in (0, len(pairs))
    for q in range(ns):
        i, j = pairs[q]
        assert np.array_equal(planes[L + q], planes[i] + planes[j])
        assert np.all(np.abs(planes[L + q]) <= 256)


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("n,k", [(2, 4), (66, 132), (130, 260), (96, 40)])
def test_sblocks_match_oracle(p, n, k):
    from paper_2101_01025_gb300 import testing as T
    kind, a, b = T.y_params(p)
    if kind == 2 and (k // 2) % 2:
        pytest.skip("kind-2 Y needs k/2 even")
    A = synth.residues(n * 1000 + k, (n, k), p)
    got = [host(s) for s in T.sblocks(dev(A), p)]
    ref = oracle.alg1_sblocks(A, p, kind, a, b)
    for i in range(4):
        assert np.array_equal(got[i].astype(np.int64), ref[i].astype(np.int64)), "S%d" % (i + 1)


LEAFKINDS = {"tc": 0, "tc_plain": 1 << 12, "simt": 1 << 4, "i8": 2 << 4, "f64": 3 << 4}


@pytest.mark.parametrize("leafkind", list(LEAFKINDS))
@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 520, 200), (1000, 700, 1536),
                                   (5, 3, 1), (257, 129, 777), (640, 512, 9000)])
def test_leaf_gemm_matches_oracle(leafkind, p, M, N, K):
    from paper_2101_01025_gb300 import testing as T
    if leafkind == "simt" and K > 2000:
        pytest.skip("slow check path")
    if leafkind == "f64" and p == 2**31 - 1:
        with pytest.raises(Exception):      # ((p-1)/2)^2 K would round in FP64
            T.leaf(dev(np.zeros((M, K), np.int32)), dev(np.zeros((N, K), np.int32)), p,
                   leafkind=LEAFKINDS[leafkind])
        return
    kindflag = LEAFKINDS[leafkind]
    X = synth.residues(M + 7 * K, (M, K), p, balanced=True)
    Y = synth.residues(N + 11 * K, (N, K), p)
    C = host(T.leaf(dev(X), dev(Y), p, leafkind=kindflag))
    assert np.array_equal(C.astype(np.int64), oracle.gemm_modp(X, Y, p).astype(np.int64))


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("n,K", [(640, 384), (129, 1100), (1, 5)])
def test_leaf_syrk_lower_and_accumulate(p, n, K):
    from paper_2101_01025_gb300 import testing as T
    X = synth.residues(n * 3 + K, (n, K), p)
    Xd = dev(X)
    sentinel = -7
    C = torch.full((n, n), sentinel, dtype=torch.int32, device="cuda")
    T.leaf(Xd, Xd, p, C=C, lower=True)
    Ch = host(C)
    ref = oracle.aat_modp_low(X, p).astype(np.int64)
    assert low_equal(Ch, ref)
    assert np.all(Ch[np.triu_indices(n, 1)] == sentinel)   # upper part untouched
    # accumulate: C <- C + X X^T (lower)
    T.leaf(Xd, Xd, p, C=C, lower=True, accumulate=True)
    assert low_equal(host(C), (2 * ref) % p)


@pytest.mark.parametrize("exact_bits,scheme", [(24, 0), (23, 0), (22, 0),
                                                (24, 1 << 12), (23, 1 << 12), (20, 1 << 12)])
def test_leaf_tc_worst_case_digits_fp32_exact(exact_bits, scheme):
    """All rows equal, low digits -128 (|digit products| 2^14, one sign per
    digit pair): every FP32 partial sum of a chunk reaches exactly
    2^exact_bits before it is drained."""
    from paper_2101_01025_gb300 import testing as T
    p = 2**31 - 1
    x = -128 * (1 + 2**8 + 2**16) - 63 * 2**24
    assert abs(x) <= (p - 1) // 2
    M, N, K = 256, 512, 4096
    X = np.full((M, K), x, dtype=np.int32)
    Y = np.full((N, K), x, dtype=np.int32)
    Y[::3] = -x
    C = host(T.leaf(dev(X), dev(Y), p, leafkind=scheme, exact_bits=exact_bits)).astype(np.int64)
    pos, neg = (x * x * K) % p, (-x * x * K) % p
    assert np.all(C[:, 0::3] == neg)
    assert np.all(C[:, 1::3] == pos) and np.all(C[:, 2::3] == pos)
    ref = oracle.gemm_modp(X[:2], Y[:3], p).astype(np.int64)
    assert np.array_equal(C[:2, :3], ref)


def test_postadd_matches_definitions():
    from paper_2101_01025_gb300 import testing as T
    p = 131071
    h = 200
    C = synth.residues(5, (2 * h, 2 * h), p)
    P1, P5 = np.tril(C[:h, :h]).astype(np.int64), np.tril(C[:h, h:]).astype(np.int64)
    P3, P4T = C[h:, :h].astype(np.int64), C[h:, h:].astype(np.int64)
    U1 = P1 + P5
    U1 = np.tril(U1) + np.tril(U1, -1).T
    U2 = U1 + P4T.T
    U4 = (U2 + P3) % p
    U5 = np.tril((U2 + P4T) % p)
    got = host(T.postadd(dev(C), h, p)).astype(np.int64)
    assert np.array_equal(got[h:, :h], U4)
    assert np.array_equal(np.tril(got[h:, h:]), U5)
    assert np.array_equal(got[:h, :], C[:h, :])      # C11, C12 untouched


# ------------------------------------------------------------ whole product

SHAPES = [(1, 1), (2, 3), (17, 33), (128, 64), (256, 512), (300, 200), (513, 257),
          (640, 640), (1024, 96)]


@pytest.mark.parametrize("p", PRIMES + [13])
@pytest.mark.parametrize("n,k", SHAPES)
@pytest.mark.parametrize("levels", [0, 1, 2, 3])
def test_aat_modp_tc_matches_oracle(lib, p, n, k, levels):
    A = synth.residues(p + n * 31 + k, (n, k), p)
    C = host(lib.aat_modp(dev(A), p, levels=levels))
    assert low_equal(C, oracle.aat_modp_low(A, p))


@pytest.mark.parametrize("p", [131071, 2**31 - 1])
@pytest.mark.parametrize("n,k", [(300, 200), (256, 512), (513, 257)])
@pytest.mark.parametrize("levels", [1, 2])
def test_aat_modp_simt_leaf_matches_oracle(lib, p, n, k, levels):
    A = synth.residues(n + k, (n, k), p)
    C = host(lib.aat_modp(dev(A), p, levels=levels, flags=lib.AAT_LEAF_SIMT))
    assert low_equal(C, oracle.aat_modp_low(A, p))


@pytest.mark.parametrize("leaf", ["i8", "f64"])
@pytest.mark.parametrize("p", [65521, 131071, 2**31 - 1])
@pytest.mark.parametrize("n,k", [(300, 200), (513, 257), (256, 512)])
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_aat_modp_mma_leaves_match_oracle(lib, leaf, p, n, k, levels):
    if leaf == "f64" and p == 2**31 - 1:
        pytest.skip("no exact FP64 leaf for this p (checked on the host)")
    A = synth.residues(5 * n + k + levels, (n, k), p)
    C = host(lib.aat_modp(dev(A), p, levels=levels, flags=LEAFKINDS[leaf]))
    assert low_equal(C, oracle.aat_modp_low(A, p))


@pytest.mark.parametrize("p", [65521, 2**31 - 1, 1000003, 13])
@pytest.mark.parametrize("n,k", [(1, 1), (17, 33), (256, 512), (300, 200), (513, 257),
                                 (640, 640), (1024, 96)])
@pytest.mark.parametrize("levels", [0, 1, 2, 3])
def test_aat_modp_low_memory_matches_oracle(lib, p, n, k, levels):
    """The low-memory schedule (one plane of each operand per pass, products
    accumulated in C) is bit-exact at every depth, ragged and k > n shapes,
    both kinds of Y (65521 = 1 mod 4; 2^31 - 1, 1000003 = 3 mod 4)."""
    A = synth.residues(p + n * 37 + k, (n, k), p)
    C = host(lib.aat_modp(dev(A), p, levels=levels, flags=lib.AAT_LOW_MEMORY))
    assert low_equal(C, oracle.aat_modp_low(A, p))


@pytest.mark.parametrize("width", [2, 3, 4])
def test_aat_modp_low_memory_plane_windows(lib, monkeypatch, width):
    """Passes over windows of 2, 3 or 4 planes (the last window narrower),
    at 1 and 2 levels over F_{2^31-1}."""
    monkeypatch.setenv("AAT_PASS_PLANES", str(width))
    p = 2**31 - 1
    for levels, (n, k) in ((1, (640, 512)), (2, (520, 780))):
        A = synth.residues(width * 100 + levels, (n, k), p, balanced=True)
        C = host(lib.aat_modp(dev(A), p, levels=levels, flags=lib.AAT_LOW_MEMORY))
        assert low_equal(C, oracle.aat_modp_low(A, p))


def test_workspace_limit_selects_low_memory(lib):
    """A workspace limit below the fast schedule's need runs the low-memory
    schedule (same result); an allocation failure of the fast workspace falls
    back to it too; below the low-memory need the call reports AAT_ENOMEM."""
    from paper_2101_01025_gb300 import _native
    p = 2**31 - 1
    n, k = 1024, 768
    A = synth.residues(99, (n, k), p, balanced=True)
    ref = oracle.aat_modp_low(A, p)
    fast = lib.aat_workspace_size(n, k, p, lib.AAT_LEVELS(1))
    low = lib.aat_workspace_size(n, k, p, lib.AAT_LEVELS(1) | lib.AAT_LOW_MEMORY)
    assert low * 4 <= fast
    nat = _native.lib()
    try:
        lib.aat_set_workspace_limit(low)
        assert lib.aat_workspace_size(n, k, p, lib.AAT_LEVELS(1)) == low
        assert low_equal(host(lib.aat_modp(dev(A), p, levels=1)), ref)
    finally:
        lib.aat_set_workspace_limit(None)
    lib.aat_shutdown()
    try:
        nat.aatx_set_alloc_limit(low)           # the fast workspace cannot be had
        assert low_equal(host(lib.aat_modp(dev(A), p, levels=1)), ref)
        nat.aatx_set_alloc_limit(low // 2)      # nor the low-memory one
        with pytest.raises(lib.AatError) as ei:
            lib.aat_modp(dev(A), p, levels=1)
        assert ei.value.code == _native.AAT_ENOMEM
    finally:
        nat.aatx_set_alloc_limit(2**64 - 1)


@pytest.mark.parametrize("leaf", ["tc", "i8", "f64"])
def test_config1_512_p131071_one_level_every_leaf(lib, leaf):
    """The small workload exactly: A 512 x 512 over F_131071 (131071 = 3 mod 4,
    so Y = [[a, b], [-b, a]] (x) I), uniform residues in [0, p) from the
    seeded generator, one recursion level then the leaf, bit-exact against the
    oracle with each of the three leaf kinds."""
    p, n = 131071, 512
    A = synth.residues(synth.SEED_BASE + 0, (n, n), p)
    C = host(lib.aat_modp(dev(A), p, levels=1, flags=LEAFKINDS[leaf]))
    assert low_equal(C, oracle.aat_modp_low(A, p))
    from paper_2101_01025_gb300 import testing as T
    st = T.plan_stats(n, n, p, lib.AAT_LEVELS(1) | LEAFKINDS[leaf])
    assert st.levels == 1 and st.n_pad == n and st.k_pad == n
    assert st.recursive_products == 3 and st.general_products == 2 and st.syrk_leaves == 3


@pytest.mark.parametrize("p", [65521, 2**31 - 1])
@pytest.mark.parametrize("n,k", [(300, 200), (640, 640)])
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_aat_modp_plain_digit_pairs_matches_oracle(lib, p, n, k, levels):
    A = synth.residues(7 * n + k, (n, k), p)
    C = host(lib.aat_modp(dev(A), p, levels=levels, flags=lib.AAT_DIGITS_PLAIN))
    assert low_equal(C, oracle.aat_modp_low(A, p))


def test_aat_modp_strides_balanced_zero_upper(lib):
    p = 2**31 - 1
    n, k = 384, 256
    big = synth.residues(9, (n, k + 40), p, balanced=True)
    Ad = dev(big)[:, 13:13 + k]                        # lda = k + 40
    Cbig = torch.full((n, n + 24), 5, dtype=torch.int32, device="cuda")
    Cd = Cbig[:, 8:8 + n]                              # ldc = n + 24
    lib.aat_modp(Ad, p, C=Cd, levels=2, flags=lib.AAT_ZERO_UPPER | lib.AAT_IN_BALANCED)
    got = host(Cbig)
    ref = oracle.aat_modp_low(np.ascontiguousarray(big[:, 13:13 + k]), p)
    assert low_equal(got[:, 8:8 + n], ref)
    assert np.all(got[:, 8:8 + n][np.triu_indices(n, 1)] == 0)
    assert np.all(got[:, :8] == 5) and np.all(got[:, 8 + n:] == 5)


def test_aat_modp_empty_and_degenerate(lib):
    p = 131071
    C = torch.full((3, 3), 9, dtype=torch.int32, device="cuda")
    lib.aat_modp(torch.zeros((3, 0), dtype=torch.int32, device="cuda"), p, C=C)
    assert np.all(np.tril(host(C)) == 0)
    lib.aat_modp(torch.zeros((0, 5), dtype=torch.int32, device="cuda"), p)
    A = np.zeros((64, 64), dtype=np.int32)
    A[np.arange(64), np.arange(64)] = 1
    assert low_equal(host(lib.aat_modp(dev(A), p, levels=2)), np.eye(64))


@pytest.mark.parametrize("p", PRIMES)
def test_aat_gemm_modp_matches_oracle(lib, p):
    X = synth.residues(3, (333, 450), p)
    Y = synth.residues(4, (270, 450), p)
    C = host(lib.aat_gemm_modp(dev(X), dev(Y), p))
    assert np.array_equal(C.astype(np.int64), oracle.gemm_modp(X, Y, p).astype(np.int64))
    F = host(lib.aat_gemm_modp(dev(X), dev(X), p))
    assert np.array_equal(F.astype(np.int64), oracle.gemm_modp(X, X, p).astype(np.int64))


def test_aat_modp_host_end_to_end(lib):
    p = 65521
    A = synth.residues(77, (700, 900), p)
    C = lib.aat_modp_host(A, p)
    assert low_equal(C, oracle.aat_modp_low(A, p))


@pytest.mark.parametrize("levels", [1, 2])
def test_aat_modp_host_early_rows_overlap(lib, levels):
    """Pinned buffers, a recursion level: rows below n/2 are copied back on a
    second stream while the last product runs; the lower triangle must equal
    the device path's and sampled oracle entries (band edges, the split)."""
    p = 2**31 - 1
    n, k = 1536, 1024
    A = synth.residues(91, (n, k), p, balanced=True)
    Ah = torch.from_numpy(A).pin_memory()
    Ch = torch.full((n, n), -7, dtype=torch.int32).pin_memory()
    lib.aat_modp_host(Ah, p, C=Ch, levels=levels)
    got = Ch.numpy()
    ref_dev = host(lib.aat_modp(dev(A), p, levels=levels))
    assert low_equal(got, ref_dev)
    rows = sorted({0, 1, 511, 512, 513, n // 2 - 1, n // 2, n // 2 + 1, 1023, 1024, n - 1})
    ij = np.array([(i, j) for i in rows for j in sorted({0, i // 2, i})], dtype=np.int64)
    ref = oracle.aat_modp_entries(A, p, ij)
    assert np.array_equal(got[ij[:, 0], ij[:, 1]].astype(np.int64), np.asarray(ref, dtype=np.int64))


def test_autotune_choice_is_used_and_exact(lib):
    """aat_tune_modp times every candidate (levels, leaf form, digit form)
    for one shape; later calls of that shape take the choice from the table
    and stay bit-exact."""
    p = 2**31 - 1
    n, k = 2048, 1024
    lib.tune_clear()
    t = lib.tune_modp(n, k, p, reps=1)
    assert t["form"] in (0, 1, 2) and 0 <= t["levels"] <= 4 and t["plain_digits"] in (0, 1)
    assert t["ms"] > 0 and t["ms_default"] > 0
    assert lib.tune_lookup(n, k, p) == t
    from paper_2101_01025_gb300 import testing as T
    assert T.plan_stats(n, k, p).levels == t["levels"]
    A = synth.residues(93, (n, k), p, balanced=True)
    C = host(lib.aat_modp(dev(A), p))
    ref = host(lib.aat_modp(dev(A), p, levels=1))
    assert low_equal(C, ref)
    ij = np.array([(i, j) for i in (0, 1, 1023, 1024, 2047) for j in (0, i // 3, i)],
                  dtype=np.int64)
    want = np.asarray(oracle.aat_modp_entries(A, p, ij), dtype=np.int64)
    assert np.array_equal(C[ij[:, 0], ij[:, 1]].astype(np.int64), want)
    lib.tune_clear()


def test_aat_modp_host_zero_upper_copies_everything(lib):
    p = 131071
    A = synth.residues(92, (600, 400), p)
    C = np.full((600, 600), 5, dtype=np.int32)
    lib.aat_modp_host(A, p, C=C, flags=lib.AAT_ZERO_UPPER, levels=1)
    assert low_equal(C, oracle.aat_modp_low(A, p))
    assert not np.triu(C, 1).any()


# -------------------------------------------------------- full-size cases

def _sample_pairs(n, levels, count, seed):
    """Random lower entries plus every recursion block boundary +-1 and the
    diagonal near them."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, n, count)
    j = rng.integers(0, n, count)
    pairs = [(max(a, b), min(a, b)) for a, b in zip(i, j)]
    edges = set()
    for lv in range(1, levels + 1):
        step = n >> lv
        for e in range(0, n + 1, step):
            for d in (-1, 0):
                if 0 <= e + d < n:
                    edges.add(e + d)
    edges = sorted(edges)
    for a in edges:
        for b in edges:
            if b <= a:
                pairs.append((a, b))
    return np.array(pairs, dtype=np.int64)


def _full_check(lib, A, p, levels_expected_min=1, nsample=3000, nvec=2, levels=None, flags=0):
    """levels None: the default launch configuration (as bench.py)."""
    from paper_2101_01025_gb300 import _native
    from paper_2101_01025_gb300 import testing as T
    n, k = A.shape
    lvf = 0 if levels is None else _native.AAT_LEVELS(levels)
    st = T.plan_stats(n, k, p, lvf | flags)
    assert st.levels >= levels_expected_min
    C = lib.aat_modp(dev(A), p, levels=levels, flags=flags)
    Ch = host(C)
    del C
    ij = _sample_pairs(n, st.levels, nsample, seed=n + k)
    ref = oracle.aat_modp_entries(A, p, ij)
    got = Ch[ij[:, 0], ij[:, 1]].astype(np.int64)
    assert np.array_equal(got, ref.astype(np.int64))
    xs = synth.vectors_mod_p(1234, nvec, n, p)
    assert oracle.freivalds_modp(A, Ch, p, xs) == 0
    return st


@functools.lru_cache(maxsize=1)
def _bench_input():
    return synth.residues(synth.SEED_BASE + 2, (16384, 16384), 2**31 - 1, balanced=True)


def test_full_size_n16384_p2_31m1(lib):
    p = 2**31 - 1
    st = _full_check(lib, _bench_input(), p, levels_expected_min=1)
    assert st.n_pad == 16384


def test_full_size_n16384_p2_31m1_winograd(lib):
    """The bench workload with Winograd's form for the last level's P3, P4."""
    p = 2**31 - 1
    st = _full_check(lib, _bench_input(), p, levels_expected_min=1, flags=lib.AAT_WINOGRAD)
    assert st.general_products == 14 * 3 ** (st.levels - 1) + 2 * (3 ** (st.levels - 1) - 1) // 2


def test_full_size_n16384_p2_31m1_low_memory(lib):
    """The bench workload on the low-memory schedule (S blocks in C, plane
    passes; at most A's size of workspace instead of 8.75 GiB): sampled
    entries and Freivalds."""
    p = 2**31 - 1
    assert lib.aat_workspace_size(16384, 16384, p, lib.AAT_LOW_MEMORY) <= 4 * 16384 * 16384
    st = _full_check(lib, _bench_input(), p, levels_expected_min=1, flags=lib.AAT_LOW_MEMORY)
    assert st.n_pad == 16384


@functools.lru_cache(maxsize=4)
def _config2_input(n, k, p):
    return synth.residues(synth.SEED_BASE + 1, (n, k), p)


@pytest.mark.parametrize("levels", [None, 2, 3])
@pytest.mark.parametrize("n,k,p", [(8192, 8192, 65521), (8192, 8192, 131071),
                                   (16384, 4096, 65521), (16384, 4096, 131071)])
def test_full_size_config2(lib, n, k, p, levels):
    """8192 x 8192 and 16384 x 4096 over F_65521 and F_131071 with the default
    depth and with 2 and 3 recursion levels: sampled entries and Freivalds."""
    A = _config2_input(n, k, p)
    st = _full_check(lib, A, p, levels_expected_min=0, nsample=1500, nvec=1, levels=levels)
    if levels is not None:
        assert st.levels == levels


@pytest.mark.parametrize("leaf", ["i8", "f64"])
@pytest.mark.parametrize("n,k,p", [(8192, 8192, 65521), (16384, 4096, 131071)])
def test_full_size_config2_mma_leaves(lib, leaf, n, k, p):
    """The INT8 and FP64 mma.sync leaves at full size with 2 levels: sampled
    entries and Freivalds, bit-exact like the BF16-digit leaf."""
    A = _config2_input(n, k, p)
    st = _full_check(lib, A, p, levels_expected_min=2, nsample=800, nvec=1, levels=2,
                     flags=LEAFKINDS[leaf])
    assert st.levels == 2


# ------------------------------------------------------- SYRK form (Sec. 7)

@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("n,k,levels", [(512, 384, 1), (600, 400, 2), (333, 250, 1),
                                        (256, 640, 1), (700, 350, 0)])
def test_syrk_update_matches_oracle(lib, p, n, k, levels):
    """Low(C) <- alpha Low(A A^T) + beta Low(C) by the Table 4 schedule:
    ragged and padded shapes, k > n (S3 in workspace), 0-2 levels."""
    A = synth.residues(51, (n, k), p, balanced=(p == 2**31 - 1))
    C0 = synth.residues(52, (n, n), p).astype(np.int32)
    for alpha, beta in [(1, 1), (7, p - 3), (p - 1, 2**32 - 5)]:
        C = dev(C0)
        lib.aat_syrk_modp(alpha, dev(A), beta, C, p, levels=levels)
        want = oracle.syrk_modp_low(alpha, A, beta % p, C0, p)
        assert low_equal(host(C), want), (alpha, beta)


@pytest.mark.parametrize("leaf", ["AAT_LEAF_SIMT", "AAT_LEAF_I8"])
def test_syrk_update_other_leaves(lib, leaf):
    p = 131071
    A = synth.residues(53, (384, 256), p)
    C0 = synth.residues(54, (384, 384), p).astype(np.int32)
    C = dev(C0)
    lib.aat_syrk_modp(5, dev(A), 9, C, p, flags=getattr(lib, leaf), levels=2)
    assert low_equal(host(C), oracle.syrk_modp_low(5, A, 9, C0, p))


def test_syrk_update_degenerate(lib):
    p = 65521
    A = synth.residues(55, (300, 200), p)
    C0 = synth.residues(56, (300, 300), p).astype(np.int32)
    # beta = 0: alpha times the product; alpha = 0: beta C; k = 0: beta C
    C = dev(C0)
    lib.aat_syrk_modp(3, dev(A), 0, C, p)
    assert low_equal(host(C), oracle.syrk_modp_low(3, A, 0, C0, p))
    C = dev(C0)
    lib.aat_syrk_modp(0, dev(A), 4, C, p)
    assert low_equal(host(C), oracle.syrk_modp_low(0, A, 4, C0, p))
    C = dev(C0)
    lib.aat_syrk_modp(2, torch.empty((300, 0), dtype=torch.int32, device="cuda"), 6, C, p)
    assert low_equal(host(C), (6 * C0.astype(np.int64)) % p)
    # balanced C entries on input, zeroed upper triangle on request
    Cb = np.where(C0 > p // 2, C0 - p, C0).astype(np.int32)
    C = dev(Cb)
    lib.aat_syrk_modp(1, dev(A), 1, C, p, flags=lib.AAT_ZERO_UPPER, levels=1)
    got = host(C)
    assert low_equal(got, oracle.syrk_modp_low(1, A, 1, C0, p))
    assert not np.triu(got, 1).any()


@pytest.mark.parametrize("p", [1000003, 2147483587])
@pytest.mark.parametrize("levels", [1, 2])
def test_p_3_mod_8_y_with_a_equal_one(lib, p, levels):
    """p = 3 mod 8 takes Y = [[1, sqrt(-2)], [-sqrt(-2), 1]] (x) I (Lemma 4.3):
    the result is the same Low(A A^T) mod p."""
    A = synth.residues(61, (520, 456), p, balanced=True)
    C = host(lib.aat_modp(dev(A), p, levels=levels))
    assert low_equal(C, oracle.aat_modp_low(A, p))


# --------------------------------------------------- quaternions (Sec. 6.2)

@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("n,k,levels", [(300, 257, 1), (512, 384, 2), (129, 70, 0)])
def test_quaternion_aah_matches_oracle(lib, p, n, k, levels):
    """M M^H for M = A + B i + C j + D k by the 6-multiplication algorithm:
    the four lower triangles, bit-exact, ragged and padded shapes."""
    parts = [synth.residues(100 + q, (n, k), p, balanced=(q % 2 == 1)) for q in range(4)]
    H = lib.aah_quat_modp(*[dev(X) for X in parts], p, levels=levels)
    want = oracle.quat_aah_modp_low(*parts, p)
    for q in range(4):
        assert low_equal(host(H[q]), want[q]), q


def test_quaternion_aah_other_leaf_and_zero_upper(lib):
    p = 131071
    parts = [synth.residues(110 + q, (200, 160), p) for q in range(4)]
    H = lib.aah_quat_modp(*[dev(X) for X in parts], p, flags=lib.AAT_LEAF_SIMT | lib.AAT_ZERO_UPPER,
                          levels=1)
    want = oracle.quat_aah_modp_low(*parts, p)
    for q in range(4):
        got = host(H[q])
        assert low_equal(got, want[q]) and not np.triu(got, 1).any()


_FORM_SCRIPT = r"""
import sys
import numpy as np
import torch
import oracle
import paper_2101_01025_gb300 as aat
from paper_2101_01025_gb300 import synth
for p in (65521, 2**31 - 1):
    for n, k, levels in ((1536, 1024, 1), (1024, 2048, 2), (520, 264, 1)):
        A = synth.residues(n * 3 + k + p % 97, (n, k), p)
        C = aat.aat_modp(torch.from_numpy(A).cuda(), p, levels=levels)
        torch.cuda.synchronize()
        got = np.tril(C.cpu().numpy().astype(np.int64))
        ref = np.tril(np.asarray(oracle.aat_modp_low(A, p), dtype=np.int64))
        if not np.array_equal(got, ref):
            print("MISMATCH", p, n, k, levels)
            sys.exit(1)
assert aat.aat_device_status() == 0
print("OK")
"""


@pytest.mark.parametrize("env", [{"AAT_LEAF_FUSE": "0"}, {"AAT_LEAF_PAIR": "1"},
                                 {"AAT_LEAF_PAIR": "0"}])
def test_leaf_launch_forms(env):
    """The last level's four independent products run as one launch by
    default; the same results with one launch per product (AAT_LEAF_FUSE=0)
    and with every leaf forced onto the CTA-pair or the one-CTA form (these
    switches are read once per process, so each runs in a child process)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FORM_SCRIPT], cwd=root,
                       env={**os.environ, **env}, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "OK" in r.stdout, r.stdout + r.stderr


# ------------------------------------- Winograd's form for P3 and P4 (Thm 3.1)

@pytest.mark.parametrize("p", PRIMES + [13])
@pytest.mark.parametrize("n,k", [(8, 8), (300, 200), (256, 512), (640, 640), (1024, 2048),
                                 (1032, 520), (513, 257)])
@pytest.mark.parametrize("levels", [1, 2])
def test_aat_modp_winograd_matches_oracle(lib, p, n, k, levels):
    """AAT_WINOGRAD: the last level's general products by Winograd's form
    (ragged quarter blocks, k > n, padded shapes, both kinds of Y)."""
    A = synth.residues(11 * n + k + levels, (n, k), p)
    C = host(lib.aat_modp(dev(A), p, levels=levels, flags=lib.AAT_WINOGRAD))
    assert low_equal(C, oracle.aat_modp_low(A, p))


def test_aat_modp_winograd_host_path(lib):
    """The end-to-end path (P1 computed while the rest of A arrives) with
    Winograd's form."""
    p = 2**31 - 1
    A = synth.residues(17, (1536, 1024), p, balanced=True)
    C = lib.aat_modp_host(A, p, levels=1, flags=lib.AAT_WINOGRAD)
    assert low_equal(C, oracle.aat_modp_low(A, p))
