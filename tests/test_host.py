"""Host logic of the library, no GPU needed: the C ABI loads and exports every
declared symbol, the host number theory, the digit split plan, the
recursion plan against the paper's counts, and argument validation."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2101_01025_gb300 import _native, build as buildmod, testing as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    buildmod.build()
    yield


def _declared_symbols():
    names = set()
    for h in ("aat.h", "aat_testing.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        names.update(re.findall(r"AAT_API\s+[\w\s\*]+?\b(aa[a-z]*_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = _native.lib()
    declared = _declared_symbols()
    assert declared == set(_native.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
    assert lib.aat_version() >= 100


def test_number_theory_matches_definitions():
    for p in [3, 5, 7, 11, 13, 97, 65521, 131071, 131041, 2**31 - 1]:
        assert T.is_prime(p)
    for q in [1, 4, 9, 65521 * 3, 2**31 - 3, 3215031751]:
        assert not T.is_prime(q)
    s = np.ones(3000, dtype=bool)
    s[:2] = False
    for i in range(2, 60):
        s[i * i::i] = False
    for q in range(3000):
        assert T.is_prime(q) == bool(s[q])
    for p in [3, 7, 13, 17, 101, 65521, 131071, 2**31 - 1]:
        for a in range(0, min(p, 300)):
            r = T.sqrt_mod(a, p)
            if r is None:
                assert oracle.legendre(a, p) == -1
            else:
                assert (r * r - a) % p == 0


@pytest.mark.parametrize("p", [3, 5, 7, 11, 13, 65521, 131071, 131041, 2**31 - 1])
def test_y_is_skew_unitary(p):
    """The library's Y satisfies Y Y^T = -I (Eq. skewu), independently of the
    oracle's choice of root (which may differ: any skew-unitary Y works)."""
    kind, a, b = T.y_params(p)
    if p % 4 == 1:
        assert kind == 1 and (a * a + 1) % p == 0
    else:
        assert kind == 2 and (a * a + b * b + 1) % p == 0
    Y = oracle.build_y(kind, a, b, p, 6).astype(object)
    assert np.array_equal((Y @ Y.T) % p, (np.eye(6, dtype=object) * (p - 1)) % p)


@pytest.mark.parametrize("p", [3, 11, 19, 43, 59, 83, 1000003, 2147483587])
def test_y_has_a_equal_one_when_p_is_3_mod_8(p):
    """p = 3 mod 8: Lemma 4.3 makes -2 a square, so the library takes a = 1,
    b = sqrt(-2) (two multiplications by Y entries per column pair instead
    of three, the examples closing Sec. 3)."""
    assert p % 8 == 3 and oracle.is_prime(p)
    kind, a, b = T.y_params(p)
    assert kind == 2 and a == 1 and (1 + b * b) % p == p - 1


def test_y_cache_many_primes():
    """Y is kept per prime after its first computation: for 300 primes (all
    three kinds of Y), a second request returns the first answer, and every
    answer is skew-unitary."""
    primes = [q for q in range(3, 200000) if oracle.is_prime(q)][-300:]
    first = {q: T.y_params(q) for q in primes}
    for q in primes:
        kind, a, b = T.y_params(q)
        assert (kind, a, b) == first[q]
        if q % 4 == 1:
            assert kind == 1 and (a * a + 1) % q == 0
        else:
            assert kind == 2 and (a * a + b * b + 1) % q == 0
    assert {q % 8 for q in primes} >= {1, 3, 5, 7}


def test_sos_all_residues():
    for p in [3, 7, 11, 19, 23, 131071]:
        for k in list(range(min(p, 200))) + [p - 1]:
            a, b = T.sos(k, p)
            assert (a * a + b * b - k) % p == 0


def _digits(x, b, L):
    """The balanced base-2^b digit rule applied to one integer (Python)."""
    out = []
    half = 1 << (b - 1)
    for _ in range(L - 1):
        d = ((x + half) & ((1 << b) - 1)) - half
        out.append(d)
        x = (x - d) >> b
    out.append(x)
    return out


@pytest.mark.parametrize("p", [3, 13, 257, 65521, 131071, 131041, 2**31 - 1])
def test_digit_spec_bounds_and_exactness(p):
    b, L, dmax = T.digit_spec(p)
    half = (p - 1) // 2
    vals = [0, 1, -1, half, -half, half - 1, -(half - 1)]
    rng = np.random.default_rng(p)
    vals += [int(v) for v in rng.integers(-half, half + 1, 2000)]
    for x in vals:
        ds = _digits(x, b, L)
        assert sum(d << (b * i) for i, d in enumerate(ds)) == x
        for i, d in enumerate(ds):
            assert abs(d) <= dmax[i], (x, ds, dmax)
            assert abs(d) <= 256      # exact in bfloat16
    # the worst case is reached: every bound is attained by some x
    assert max(dmax) ** 2 <= 1 << 16
    if p == 2**31 - 1:
        assert (b, L) == (8, 4)
    if p in (65521, 131071):
        assert L == 2
    # pair sums are used exactly when every d_i + d_j stays within 256
    ns = T.digit_spec(p, with_sums=True)[3]
    ok = 2 <= L <= 4 and all(dmax[i] + dmax[j] <= 256 for i in range(L) for j in range(i + 1, L))
    assert ns == (L * (L - 1) // 2 if ok else 0)
    if p == 2**31 - 1:
        assert ns == 6          # 10 plane products instead of 16
    if p == 131071:
        assert ns == 0          # d_1 reaches 256: plain pairs


def test_plan_counts_match_paper():
    """Each level has 3 recursive products, 2 general products and 9 block
    additions, 3 of them on symmetric blocks (Alg. 1; Remark 3.3); the ring
    MACs follow s(l) = 3/8 s(l-1) + 1/4 with s(0) = 1/2 (Table 1)."""
    p = 2**31 - 1
    n = k = 16384
    s = 0.5
    for lv in range(0, 5):
        st = T.plan_stats(n, k, p, _native.AAT_LEVELS(lv))
        nodes = sum(3 ** i for i in range(lv))       # internal nodes
        assert st.levels == lv
        assert st.recursive_products == 3 * nodes
        assert st.block_additions == 9 * nodes
        assert st.half_additions == 3 * nodes
        assert st.general_products == 2 * nodes
        assert st.syrk_leaves == 3 ** lv
        leading = st.ring_macs / (n * n * k)
        assert abs(leading - s) < 2.0 / (n >> lv), (lv, leading, s)
        s = 3.0 / 8.0 * s + 0.25
    st = T.plan_stats(n, k, p)
    assert st.levels >= 1      # the automatic choice recurses at this size


def test_plan_padding_and_workspace():
    p = 131071
    st = T.plan_stats(1001, 333, p, _native.AAT_LEVELS(2))
    assert st.n_pad == 1004 and st.k_pad % 8 == 0 and st.k_pad >= 333
    st0 = T.plan_stats(1001, 333, p, _native.AAT_LEVELS(0))
    assert st0.n_pad == 1001 and st0.k_pad == 333
    lib = _native.lib()
    assert lib.aat_workspace_size(16384, 16384, 2**31 - 1, 0) > 0
    assert lib.aat_workspace_size(0, 10, 131071, 0) == 0


def test_argument_validation_before_any_gpu_call():
    lib = _native.lib()
    fake = 1 << 20   # never dereferenced: validation fails first
    assert lib.aat_modp_ex(fake, 4, 4, 4, 15, fake * 2, 4, 0, None) == _native.AAT_ENOTPRIME
    assert lib.aat_modp_ex(fake, 4, 4, 4, 2, fake * 2, 4, 0, None) == _native.AAT_ENOTPRIME
    assert lib.aat_modp_ex(fake, 4, 4, 4, 2147483659, fake * 2, 4, 0, None) == _native.AAT_ERANGE
    assert lib.aat_modp_ex(fake, -1, 4, 4, 131071, fake * 2, 4, 0, None) == _native.AAT_EINVAL
    assert lib.aat_modp_ex(fake, 4, 4, 3, 131071, fake * 2, 4, 0, None) == _native.AAT_EINVAL
    assert lib.aat_modp_ex(None, 4, 4, 4, 131071, fake * 2, 4, 0, None) == _native.AAT_EINVAL
    assert lib.aat_modp_ex(fake, 4, 4, 4, 131071, fake + 8, 4, 0, None) == _native.AAT_EINVAL
    assert "overlap" in _native.last_error()
    assert lib.aat_gemm_modp(fake, 4, fake, 4, 4, 4, 4, 9, fake * 2, 4, 0, None) == \
        _native.AAT_ENOTPRIME
    assert lib.aat_modp_ex(fake, 4, 4, 4, 131071, fake * 2, 4, 7 << 4, None) == \
        _native.AAT_EUNSUPPORTED
    # the FP64 leaf is exact only while ((p-1)/2)^2 sums stay below 2^53
    assert lib.aat_modp_ex(fake, 4, 4, 4, 2**31 - 1, fake * 2, 4, _native.AAT_LEAF_F64, None) == \
        _native.AAT_ERANGE


@pytest.mark.parametrize("p", [2**31 - 1, 65521, 131071, 13, 1000003])
@pytest.mark.parametrize("K", [1, 64, 1000, 8192, 20000])
@pytest.mark.parametrize("plain", [False, True])
def test_leaf_group_plan_reproduces_the_product(p, K, plain):
    """Simulate the leaf epilogue on random digits: per group the exact
    integer sum over its K range, Horner ratios between groups; the result
    must be sum_k x_k y_k mod p.  Also checks the FP32 and int32 bounds."""
    b, L, dmax, ns = T.digit_spec(p, with_sums=True)
    groups, nprod = T.leaf_groups(p, K, _native.AAT_DIGITS_PLAIN if plain else 0)
    use_sums = ns > 0 and not plain
    assert nprod == (L + ns if use_sums else L * L)
    pairs = [(i, j) for i in range(L) for j in range(i + 1, L)]
    rng = np.random.default_rng(p + K)
    half = (p - 1) // 2
    x = [int(v) for v in rng.integers(-half, half + 1, K)]
    y = [int(v) for v in rng.integers(-half, half + 1, K)]
    x[0], y[0] = -half, half
    dx = [_digits(v, b, L) for v in x]
    dy = [_digits(v, b, L) for v in y]

    def plane(d, q):
        return d[q] if q < L else d[pairs[q - L][0]] + d[pairs[q - L][1]]

    pmax = dmax + [dmax[i] + dmax[j] for i, j in pairs]
    acc = 0
    for gi, (xp, yp, kb0, kb1, kc, ratio) in enumerate(groups):
        if gi > 0:
            acc = acc * ratio % p
            acc = acc - p if acc > half else acc
        prod = pmax[xp] * pmax[yp]
        assert kc * 64 * prod <= 1 << 24            # FP32 partial sums stay exact
        assert half + (kb1 - kb0) * 64 * prod < 2**31  # int32 accumulator
        for k0 in range(kb0 * 64, min(kb1 * 64, K), kc * 64):
            chunk = sum(plane(dx[k], xp) * plane(dy[k], yp)
                        for k in range(k0, min(k0 + kc * 64, kb1 * 64, K)))
            assert abs(chunk) <= 1 << 24
            acc += chunk
        assert abs(acc) < 2**31
    assert acc % p == sum(a * c for a, c in zip(x, y)) % p


def test_host_copy_volume_is_the_lower_triangle_in_bands():
    """aat_modp_host copies back only the lower triangle, in bands of 512
    rows (band [a, b) carries columns [0, b)); with AAT_ZERO_UPPER the whole
    matrix."""
    import paper_2101_01025_gb300 as aat
    for n in (1, 7, 511, 512, 513, 1000, 16384):
        expect = 0
        for a in range(0, n, 512):
            b = min(n, a + 512)
            expect += 4 * b * (b - a)
        got = aat.aat_modp_host_d2h_bytes(n)
        assert got == expect
        assert 4 * n * (n + 1) // 2 <= got <= 4 * n * n
        assert aat.aat_modp_host_d2h_bytes(n, aat.AAT_ZERO_UPPER) == 4 * n * n
    assert aat.aat_modp_host_d2h_bytes(0) == 0


def test_tuning_table_save_load_and_lookup(tmp_path):
    """The autotuning table (no GPU needed for the table itself): entries
    loaded from JSON are looked up by (n, k, p), invalid ones are skipped, a
    saved table loads back to the same entries, and the plan of a tuned shape
    takes its recursion depth from the table unless the flags fix it."""
    import json
    import paper_2101_01025_gb300 as aat
    aat.tune_clear()
    assert aat.tune_lookup(4096, 2048, 2**31 - 1) is None
    src = tmp_path / "tune.json"
    entries = [
        {"n": 4096, "k": 2048, "p": 2**31 - 1, "levels": 3, "form": 1, "plain_digits": 0,
         "ms": 1.5, "ms_default": 2.0},
        {"n": 2048, "k": 2048, "p": 65521, "levels": 0, "form": 2, "plain_digits": 1,
         "ms": 0.5, "ms_default": 0.6},
        # invalid: not a prime, bad form
        {"n": 100, "k": 100, "p": 65535, "levels": 1, "form": 1, "plain_digits": 0,
         "ms": 1.0, "ms_default": 1.0},
        {"n": 100, "k": 100, "p": 65521, "levels": 1, "form": 7, "plain_digits": 0,
         "ms": 1.0, "ms_default": 1.0},
    ]
    lines = ['{"gpu": "", "entries": [']
    lines += ["  " + json.dumps(e) + ("," if i + 1 < len(entries) else "")
              for i, e in enumerate(entries)]
    lines.append("]}")
    src.write_text("\n".join(lines) + "\n")
    assert aat.tune_load(str(src)) == 2
    t = aat.tune_lookup(4096, 2048, 2**31 - 1)
    assert t["levels"] == 3 and t["form"] == 1 and t["plain_digits"] == 0
    assert aat.tune_lookup(2048, 2048, 65521)["plain_digits"] == 1
    assert aat.tune_lookup(100, 100, 65521) is None
    # the recursion plan follows the table; explicit levels win
    assert T.plan_stats(4096, 2048, 2**31 - 1).levels == 3
    assert T.plan_stats(4096, 2048, 2**31 - 1, flags=aat.AAT_LEVELS(1)).levels == 1
    out = tmp_path / "saved.json"
    assert aat.tune_save(str(out)) == 2
    saved = json.loads(out.read_text())
    assert sorted((e["n"], e["k"], e["p"], e["levels"]) for e in saved["entries"]) == \
        [(2048, 2048, 65521, 0), (4096, 2048, 2**31 - 1, 3)]
    aat.tune_clear()
    assert aat.tune_lookup(4096, 2048, 2**31 - 1) is None
    assert aat.tune_load(str(out)) == 2
    aat.tune_clear()
    with pytest.raises(aat.AatError):
        aat.tune_load(str(tmp_path / "missing.json"))


@pytest.mark.parametrize("p", [65521, 2**31 - 1])
@pytest.mark.parametrize("lv", [1, 2])
def test_plan_counts_with_winograd(p, lv):
    """With AAT_WINOGRAD the last level's two general products become 7
    products of half the size each: ring multiply-adds of the general
    products at that level fall to 7/8; everything else is unchanged."""
    n = k = 1024
    base = T.plan_stats(n, k, p, _native.AAT_LEVELS(lv))
    st = T.plan_stats(n, k, p, _native.AAT_LEVELS(lv) | _native.AAT_WINOGRAD)
    last_nodes = 3 ** (lv - 1)                    # nodes of the last level
    assert st.general_products == base.general_products + 12 * last_nodes
    assert st.syrk_leaves == base.syrk_leaves
    assert st.recursive_products == base.recursive_products
    h, kap = n >> lv, k >> lv
    saved = last_nodes * 2 * (h * h * kap) / 8    # 1/8 of each general product
    assert abs((base.ring_macs - st.ring_macs) - saved) < 1e-6 * base.ring_macs


def test_tuning_table_carries_winograd_choice(tmp_path):
    """A tuned shape whose entry chose Winograd's form runs its last level's
    general products as 7 products each; entries written without the key
    load as the plain form."""
    import json
    import paper_2101_01025_gb300 as aat
    aat.tune_clear()
    src = tmp_path / "tune.json"
    entries = [
        {"n": 1024, "k": 1024, "p": 131071, "levels": 1, "form": 0, "plain_digits": 0,
         "ms": 1.0, "ms_default": 1.1, "winograd": 1},
        {"n": 2048, "k": 1024, "p": 131071, "levels": 1, "form": 0, "plain_digits": 0,
         "ms": 1.0, "ms_default": 1.1},
        {"n": 1024, "k": 512, "p": 131071, "levels": 1, "form": 0, "plain_digits": 0,
         "ms": 1.0, "ms_default": 1.1, "winograd": 3},          # invalid
    ]
    src.write_text('{"gpu": "", "entries": [\n' +
                   ",\n".join("  " + json.dumps(e) for e in entries) + "\n]}\n")
    assert aat.tune_load(str(src)) == 2
    assert aat.tune_lookup(1024, 1024, 131071)["winograd"] == 1
    assert aat.tune_lookup(2048, 1024, 131071)["winograd"] == 0
    assert T.plan_stats(1024, 1024, 131071).general_products == 14
    assert T.plan_stats(2048, 1024, 131071).general_products == 2
    out = tmp_path / "saved.json"
    assert aat.tune_save(str(out)) == 2
    saved = {(e["n"], e["k"]): e["winograd"] for e in json.loads(out.read_text())["entries"]}
    assert saved == {(1024, 1024): 1, (2048, 1024): 0}
    aat.tune_clear()


def test_allocation_limit_hook_gives_enomem():
    """The test allocation limit turns a workspace request into AAT_ENOMEM
    before any CUDA call (so this runs without a GPU), names the request in
    the message, and SIZE_MAX lifts it again."""
    lib = _native.lib()
    try:
        lib.aatx_set_alloc_limit(1 << 20)
        assert lib.aatx_workspace_reserve((1 << 20) + 1) == _native.AAT_ENOMEM
        assert "1048577 bytes refused" in _native.last_error()
    finally:
        lib.aatx_set_alloc_limit(2**64 - 1)


def test_wait_probe_rejects_bad_arguments():
    lib = _native.lib()
    assert lib.aatx_wait_probe(2, 1000, None) == _native.AAT_EINVAL
    assert lib.aatx_wait_probe(0, 0, None) == _native.AAT_EINVAL
    assert lib.aatx_wait_probe(0, 3 * 10**9, None) == _native.AAT_EINVAL
