"""Pins of the CPU oracle to facts other than itself (run with -m "not gpu").

Each test checks the oracle against something the paper or the mathematics
fixes: closed forms, exhaustive brute force on tiny inputs, invariants,
independent library routines (numpy matmul on exact integers), and the proof
identities of Theorem 3.1.  A dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from oracle import alg1
from paper_2101_01025_gb300 import synth

SMALL_PRIMES = [3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47]
CONFIG_PRIMES = [65521, 131071, 131041, 2**31 - 1]


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")
    out = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            out[k.strip()] = float(v)
    return out


def _exact_low(A, p):
    """Low(A A^T) mod p from numpy's matmul on Python integers."""
    Ao = np.asarray(A, dtype=object) % p
    return np.tril((Ao @ Ao.T) % p).astype(np.int64)


# --------------------------------------------------------------- F_p core

@pytest.mark.parametrize("p", [3, 5, 7])
@pytest.mark.parametrize("n,k", [(1, 1), (2, 1), (1, 2), (2, 2), (3, 2), (2, 3)])
def test_low_aat_exhaustive_tiny(p, n, k):
    """Brute force: every matrix over F_p of the shape (sampled above 3^6),
    against the sum of column outer products sum_l a_l a_l^T."""
    cells = n * k
    total = p ** cells
    if total <= 20000:
        mats = itertools.product(range(p), repeat=cells)
    else:
        rng = np.random.default_rng(p * 100 + cells)
        mats = (tuple(rng.integers(0, p, cells)) for _ in range(3000))
    for vals in mats:
        A = np.array(vals, dtype=np.int32).reshape(n, k)
        C = oracle.aat_modp_low(A, p)
        ref = np.zeros((n, n), dtype=np.int64)
        for l in range(k):
            col = A[:, l].astype(np.int64)
            ref += np.outer(col, col)
        ref = np.tril(ref % p)
        assert np.array_equal(C.astype(np.int64), ref), (vals, C, ref)


@pytest.mark.parametrize("p", [131071, 65521, 2**31 - 1])
def test_low_aat_closed_forms(p):
    n, k = 9, 13
    # [I | 0] gives the identity
    A = np.zeros((n, k), dtype=np.int32)
    A[:, :n] = np.eye(n, dtype=np.int32)
    assert np.array_equal(oracle.aat_modp_low(A, p), np.eye(n, dtype=np.uint32))
    # all ones gives k everywhere (lower part)
    A = np.ones((n, k), dtype=np.int32)
    assert np.array_equal(oracle.aat_modp_low(A, p),
                          np.tril(np.full((n, n), k % p, dtype=np.uint32)))
    # Sylvester Hadamard H (entries +-1): H H^T = m I
    H = np.array([[1]], dtype=np.int64)
    for _ in range(4):
        H = np.block([[H, H], [H, -H]])
    m = H.shape[0]
    C = oracle.aat_modp_low(H.astype(np.int32), p)
    assert np.array_equal(C, (np.eye(m, dtype=np.int64) * (m % p)).astype(np.uint32))
    # rank one: A = u v^T gives (v.v) u u^T
    rng = np.random.default_rng(1)
    u = rng.integers(0, p, n).astype(object)
    v = rng.integers(0, p, k).astype(object)
    A = (np.outer(u, v) % p).astype(np.int64).astype(np.int32)
    vv = int(sum(int(x) * int(x) for x in v)) % p
    ref = np.tril((np.outer(u, u) * vv) % p).astype(np.int64)
    assert np.array_equal(oracle.aat_modp_low(A, p).astype(np.int64), ref)
    # diagonal matrix gives its square
    d = rng.integers(0, p, n)
    A = np.zeros((n, n), dtype=np.int32)
    A[np.arange(n), np.arange(n)] = d
    ref = np.diag([(int(x) * int(x)) % p for x in d]).astype(np.int64)
    assert np.array_equal(oracle.aat_modp_low(A, p).astype(np.int64), ref)


@pytest.mark.parametrize("p", [131071, 65521, 2**31 - 1, 97])
def test_low_aat_matches_exact_integers(p):
    """Against numpy matmul on exact Python integers, including entries next
    to p - 1 where (p-1)^2 k overflows 64 bits for p = 2^31 - 1."""
    rng = np.random.default_rng(p)
    for n, k in [(1, 1), (5, 3), (17, 33), (31, 64)]:
        A = rng.integers(0, p, (n, k)).astype(np.int64)
        A[0, :] = p - 1
        A = A.astype(np.int32)
        assert np.array_equal(oracle.aat_modp_low(A, p).astype(np.int64), _exact_low(A, p))


@pytest.mark.parametrize("p", [131071, 2**31 - 1])
def test_low_aat_invariants(p):
    rng = np.random.default_rng(7)
    n, k = 12, 20
    A = synth.residues(11, (n, k), p)
    C = oracle.aat_modp_low(A, p).astype(np.int64)
    # balanced representative, and adding multiples of p, change nothing
    Ab = np.where(A > p // 2, A.astype(np.int64) - p, A).astype(np.int32)
    assert np.array_equal(oracle.aat_modp_low(Ab, p).astype(np.int64), C)
    # column permutation: A P P^T A^T = A A^T (catches A^T A)
    perm = rng.permutation(k)
    assert np.array_equal(oracle.aat_modp_low(A[:, perm].copy(), p).astype(np.int64), C)
    # row permutation permutes rows and columns of the symmetric product
    rp = rng.permutation(n)
    full = C + np.tril(C, -1).T
    Cp = oracle.aat_modp_low(A[rp].copy(), p).astype(np.int64)
    assert np.array_equal(Cp, np.tril(full[np.ix_(rp, rp)]))
    # scaling row 0 by c scales row/column 0 by c and C[0,0] by c^2
    c = 12345 % p
    As = A.astype(object)
    As[0] = (As[0] * c) % p
    Cs = oracle.aat_modp_low(As.astype(np.int64).astype(np.int32), p).astype(object)
    assert Cs[0, 0] == (C[0, 0] * c * c) % p
    for i in range(1, n):
        assert Cs[i, 0] == (C[i, 0] * c) % p
        assert Cs[i, i] == C[i, i]


def test_entries_and_gemm_agree_with_definition():
    p = 131071
    A = synth.residues(5, (23, 41), p)
    C = oracle.aat_modp_low(A, p)
    ij = [(i, j) for i in range(23) for j in range(i + 1)]
    e = oracle.aat_modp_entries(A, p, ij)
    assert np.array_equal(e, np.array([C[i, j] for i, j in ij], dtype=np.uint32))
    X = synth.residues(6, (7, 41), p)
    Y = synth.residues(8, (9, 41), p)
    G = oracle.gemm_modp(X, Y, p).astype(np.int64)
    ref = ((X.astype(object) @ Y.astype(object).T) % p).astype(np.int64)
    assert np.array_equal(G, ref)
    # a general product with Y = X is the full symmetric product
    F = oracle.gemm_modp(A, A, p).astype(np.int64)
    assert np.array_equal(F, F.T)
    assert np.array_equal(np.tril(F), C.astype(np.int64))


def test_freivalds_detects_errors():
    p = 131071
    n, k = 40, 30
    A = synth.residues(3, (n, k), p)
    C = oracle.aat_modp_low(A, p).astype(np.int32)
    xs = synth.vectors_mod_p(4, 4, n, p)
    assert oracle.freivalds_modp(A, C, p, xs) == 0
    bad = C.copy()
    bad[17, 5] = (bad[17, 5] + 1) % p
    assert oracle.freivalds_modp(A, bad, p, xs) == 4
    bad = C.copy()
    bad[3, 3] = (bad[3, 3] + p - 1) % p
    assert oracle.freivalds_modp(A, bad, p, xs) == 4
    # the strict upper triangle is ignored
    up = C.copy()
    up[0, 5] = 99
    assert oracle.freivalds_modp(A, up, p, xs) == 0


# --------------------------------------------------------- number theory

def _sieve(m):
    s = np.ones(m + 1, dtype=bool)
    s[:2] = False
    for i in range(2, int(m ** 0.5) + 1):
        if s[i]:
            s[i * i::i] = False
    return s


def test_is_prime_against_sieve():
    s = _sieve(5000)
    for q in range(5001):
        assert oracle.is_prime(q) == bool(s[q]), q
    for q in CONFIG_PRIMES:
        assert oracle.is_prime(q)
    assert not oracle.is_prime(2**31 - 3)   # 2147483645 = 5 * 429496729
    assert not oracle.is_prime(65521 * 3)


def test_legendre_and_sqrt_exhaustive():
    s = _sieve(400)
    for p in [q for q in range(3, 400) if s[q]]:
        squares = {(x * x) % p for x in range(1, p)}
        assert len(squares) == (p - 1) // 2        # Euler: half the units
        for a in range(p):
            r = oracle.sqrt_mod(a, p)
            leg = oracle.legendre(a, p)
            if a == 0:
                assert leg == 0 and r == 0
            elif a in squares:
                assert leg == 1 and r is not None and (r * r) % p == a and r <= p - r
            else:
                assert leg == -1 and r is None


@pytest.mark.parametrize("p", CONFIG_PRIMES)
def test_sqrt_large_primes(p):
    rng = np.random.default_rng(p)
    for a in rng.integers(1, p, 200):
        a = int(a)
        r = oracle.sqrt_mod(a, p)
        if r is None:
            assert pow(a, (p - 1) // 2, p) == p - 1
        else:
            assert (r * r) % p == a


def test_sqrt_minus_one_exists_iff_p_1_mod_4():
    """Prop. 4.1: sqrt(-1) exists for p == 1 mod 4; (-1/p) = -1 for p == 3 mod 4."""
    s = _sieve(3000)
    for p in [q for q in range(3, 3000) if s[q]]:
        r = oracle.sqrt_mod(-1, p)
        if p % 4 == 1:
            assert r is not None and (r * r + 1) % p == 0
        else:
            assert r is None


def test_minus_two_square_for_p_3_mod_8():
    """Lemma 4.3: p == 3 mod 8 implies -2 is a square."""
    s = _sieve(5000)
    for p in [q for q in range(3, 5000) if s[q] and q % 8 == 3]:
        assert oracle.legendre(-2, p) == 1
        r = oracle.sqrt_mod(-2, p)
        assert (r * r + 2) % p == 0


def test_sos_every_k_small_primes():
    """Algorithm 3: a^2 + b^2 == k mod p for every k, every small prime."""
    for p in SMALL_PRIMES:
        for k in range(p):
            a, b = oracle.sos_modp(k, p)
            assert (a * a + b * b - k) % p == 0, (p, k, a, b)


def test_sos_minus_one_many_primes():
    s = _sieve(20000)
    for p in [q for q in range(3, 20000) if s[q]] + CONFIG_PRIMES:
        a, b = oracle.sos_modp(-1, p)
        assert (a * a + b * b + 1) % p == 0, p
        if p % 4 == 3:
            assert b != 0  # -1 is not a square there


def test_experiment_primes():
    g = _golden()
    p1 = int(g["prime_with_sqrt_minus_one"])
    p2 = int(g["prime_without_sqrt_minus_one"])
    assert oracle.is_prime(p1) and oracle.is_prime(p2)
    assert oracle.skew_unitary_params(p1)[0] == 1
    assert oracle.skew_unitary_params(p2)[0] == 2


@pytest.mark.parametrize("p", CONFIG_PRIMES + [3, 7, 13, 103])
def test_skew_unitary_y(p):
    """Eq. (skewu): Y Y^T == -I for the Y the oracle builds."""
    kind, a, b = oracle.skew_unitary_params(p)
    for kappa in (2, 4, 6, 8):
        Y = oracle.build_y(kind, a, b, p, kappa).astype(object)
        prod = (Y @ Y.T) % p
        assert np.array_equal(prod, (np.eye(kappa, dtype=object) * (p - 1)) % p)
    # the identity is not skew-unitary (negative control)
    I = np.eye(4, dtype=object)
    assert not np.array_equal((I @ I.T) % p, (np.eye(4, dtype=object) * (p - 1)) % p)


# ---------------------------------------------------------- Algorithm 1

def _alg1_cases():
    for p in [131071, 65521, 13, 2**31 - 1]:
        for (n, k) in [(8, 8), (12, 8), (8, 16), (16, 12)]:
            yield p, n, k


@pytest.mark.parametrize("p,n,k", list(_alg1_cases()))
def test_alg1_equals_definition(p, n, k):
    kind, a, b = oracle.skew_unitary_params(p)
    A = synth.residues(p % 1000 + n * 31 + k, (n, k), p)
    ref = _exact_low(A, p)
    for levels in (1, 2):
        C = alg1.alg1_low_aat(A, p, kind, a, b, levels)
        assert np.array_equal(C.astype(np.int64), ref), levels
    # the C oracle's definition agrees too
    assert np.array_equal(oracle.aat_modp_low(A, p).astype(np.int64), ref)


@pytest.mark.parametrize("p", [131071, 65521, 2**31 - 1])
def test_alg1_proof_identities(p):
    """Theorem 3.1's proof identities on the blocks of one level."""
    kind, a, b = oracle.skew_unitary_params(p)
    n, k = 12, 16
    A = synth.residues(99, (n, k), p).astype(object) % p
    tr = []
    alg1.alg1_low_aat(A, p, kind, a, b, 1, trace=tr)
    t = tr[0]
    h, kap = n // 2, k // 2
    A11, A12, A21, A22 = A[:h, :kap], A[:h, kap:], A[h:, :kap], A[h:, kap:]
    Y = t["Y"]
    md = lambda M: M % p
    eq = lambda X, Z: np.array_equal(md(X), md(Z))
    # S blocks against the C oracle's S blocks
    S = oracle.alg1_sblocks(A.astype(np.int64).astype(np.int32), p, kind, a, b)
    for name, Sc in zip(("S1", "S2", "S3", "S4"), S):
        assert eq(t[name], Sc.astype(object)), name
    # S3 = -S2 - A11 Y (proof of Thm 3.1)
    assert eq(t["S3"], -t["S2"] - A11 @ Y)
    # U3 = A11 A11^T + A12 A12^T (Low)
    assert eq(np.tril(t["U3"]), np.tril(A11 @ A11.T + A12 @ A12.T))
    R1 = A11 @ Y @ t["S2"].T
    assert eq(R1, A11 @ (Y @ A22.T + A21.T))
    S2S2 = t["S2"] @ t["S2"].T
    # U1 = S2 S2^T + R1^T + R1
    assert eq(t["U1"], S2S2 + R1.T + R1)
    R2 = A21 @ Y @ A22.T
    assert eq(S2S2, A22 @ A22.T - A21 @ A21.T - R2 - R2.T)
    assert eq(R1 + t["P4"], R2 + A21 @ A21.T)
    # U5 = A22 A22^T + A21 A21^T (Low), U4 = A22 A12^T + A21 A11^T
    assert eq(np.tril(t["U5"]), np.tril(A22 @ A22.T + A21 @ A21.T))
    assert eq(t["U4"], A22 @ A12.T + A21 @ A11.T)


def test_alg1_needs_skew_unitary_y():
    """With Y = I (Y Y^T = +I, not -I) the recursion is wrong: the
    skew-unitarity of Eq. (skewu) is what makes Algorithm 1 exact."""
    p = 131071
    A = synth.residues(5, (8, 8), p)
    wrong = alg1.alg1_low_aat(A, p, 1, 1, 0, 1)   # Y = 1 * I
    assert not np.array_equal(wrong.astype(np.int64), _exact_low(A, p))


def test_alg1_complex_transpose_and_hermitian_negative():
    """Sec. 4.1: over C, Y = i I is skew-unitary for the transposition, so
    Algorithm 1 gives A A^T; for the conjugate transposition Y Y^H = +I and
    the same recursion is wrong (no skew-unitary Y exists there)."""
    rng = np.random.default_rng(3)
    n, k = 6, 8
    A = rng.integers(-3, 4, (n, k)) + 1j * rng.integers(-3, 4, (n, k))

    def one_level(A, herm):
        adj = (lambda M: M.conj().T) if herm else (lambda M: M.T)
        h, kap = n // 2, k // 2
        A11, A12, A21, A22 = A[:h, :kap], A[:h, kap:], A[h:, :kap], A[h:, kap:]
        Y = 1j * np.eye(kap)
        S1 = (A21 - A11) @ Y
        S2 = A22 - A21 @ Y
        S3 = S1 - A22
        S4 = S3 + A12
        P1, P2 = A11 @ adj(A11), A12 @ adj(A12)
        P3, P4, P5 = A22 @ adj(S4), S1 @ adj(S2), S3 @ adj(S3)
        U1 = P1 + P5
        U2 = U1 + P4
        U4 = U2 + P3
        U5 = U2 + adj(P4)
        U3 = P1 + P2
        C = np.zeros((n, n), dtype=complex)
        C[:h, :h], C[h:, :h], C[h:, h:] = np.tril(U3), U4, np.tril(U5)
        return C

    assert np.allclose(one_level(A, False), np.tril(A @ A.T))
    assert not np.allclose(one_level(A, True), np.tril(A @ A.conj().T))


def test_alg1_cost_recurrence_constants():
    """Table 1 / Lemma 2.5: with classical products, the ring MACs of
    Algorithm 1 satisfy s(l) = 3/8 s(l-1) + 2/8 with s(0) = 1/2 (lower SYRK),
    so s(inf) = 0.4 n^3 MACs = 0.8 n^3 operations; classical D&C gives n^3."""
    g = _golden()
    s = 0.5
    for _ in range(60):
        s = 3.0 / 8.0 * s + 2.0 / 8.0
    assert abs(2 * s - g["alg1_ff_ops_over_n3"]) < 1e-12
    # Lemma (master theorem): b / (2^alpha - a) with a = 3, b = 2 MM(1) = 4
    assert abs(4.0 / (2 ** 3 - 3) - g["alg1_ff_ops_over_n3"]) < 1e-12
    assert abs(4.0 / (2 ** 3 - 4) - g["classical_ff_ops_over_n3"]) < 1e-12
    # over C: 3 real ops per complex op ... Table 2 values
    assert abs(3 * g["alg1_ff_ops_over_n3"] - g["alg1_complex_aat_ops_over_n3"]) < 1e-12
    assert abs(2 * 2.0 - g["twoM_complex_ops_over_n3"]) < 1e-12


# ------------------------------------------------------------------ C

def test_complex_oracle_exact_small_integers():
    """Small-integer complex inputs are exact in fp64: compare against Gaussian
    integer arithmetic on Python ints."""
    rng = np.random.default_rng(5)
    n, k = 7, 11
    re = rng.integers(-9, 10, (n, k))
    im = rng.integers(-9, 10, (n, k))
    A = re + 1j * im
    for conj in (True, False):
        C = oracle.complex_low(A, conj=conj)
        for i in range(n):
            for j in range(i + 1):
                sr = si = 0
                for l in range(k):
                    ar, ai = int(re[i, l]), int(im[i, l])
                    br, bi = int(re[j, l]), int(im[j, l])
                    if conj:
                        bi = -bi
                    sr += ar * br - ai * bi
                    si += ar * bi + ai * br
                assert C[i, j] == complex(sr, si)
                if conj and i == j:
                    assert si == 0 and sr >= 0


def test_complex_oracle_properties():
    A = synth.complex_normal(17, (24, 40)).astype(np.complex128)
    C = oracle.complex_low(A, conj=True)
    # Re(A A^H) = [Re Im][Re Im]^T from an independent real matmul
    RI = np.concatenate([A.real, A.imag], axis=1)
    assert np.allclose(np.tril(C.real), np.tril(RI @ RI.T), rtol=1e-12, atol=1e-10)
    assert np.allclose(np.tril(C), np.tril(A @ A.conj().T), rtol=1e-12, atol=1e-10)
    assert np.all(np.diag(C).real >= 0) and np.all(np.diag(C).imag == 0)
    # Hermitian: entry (j, i) is the conjugate of (i, j)
    ij = [(3, 7), (7, 3), (20, 1), (1, 20)]
    e = oracle.complex_entries(A, ij, conj=True)
    assert np.isclose(e[0], np.conj(e[1])) and np.isclose(e[2], np.conj(e[3]))
    # unitary DFT: F F^H = I
    m = 16
    F = np.exp(-2j * np.pi * np.outer(np.arange(m), np.arange(m)) / m) / np.sqrt(m)
    assert np.allclose(oracle.complex_low(F, conj=True), np.eye(m), atol=1e-12)
    # A A^T (no conjugation) is symmetric, not Hermitian
    T = oracle.complex_low(A, conj=False)
    assert np.allclose(np.tril(T), np.tril(A @ A.T), rtol=1e-12, atol=1e-10)


def test_two_m_algorithm():
    """Algorithm 2 (2M) returns A A^H (eps = 1) and A A^T (eps = -1)."""
    rng = np.random.default_rng(8)
    Are, Aim = rng.standard_normal((9, 13)), rng.standard_normal((9, 13))
    A = Are + 1j * Aim
    re, im = alg1.two_m(Are, Aim, conj=True)
    assert np.allclose(re + 1j * im, A @ A.conj().T)
    re, im = alg1.two_m(Are, Aim, conj=False)
    assert np.allclose(re + 1j * im, A @ A.T)


# ------------------------------------------------------------ SYRK (Sec. 7)

def _brute_syrk(alpha, A, beta, C, p):
    """alpha sum_l a_il a_jl + beta c_ij for i >= j, one entry at a time."""
    n, k = len(A), len(A[0])
    out = np.zeros((n, n), dtype=np.int64)
    for i in range(n):
        for j in range(i + 1):
            acc = beta * int(C[i][j])
            for l in range(k):
                acc += alpha * int(A[i][l]) * int(A[j][l])
            out[i, j] = acc % p
    return out


@pytest.mark.parametrize("p", [3, 5, 7])
def test_syrk_oracle_exhaustive_tiny(p):
    """Every alpha, beta and every 2 x 2 lower C with a fixed 2 x 2 A; the
    upper triangle of C must not matter (an oracle that read C^T or the upper
    part fails)."""
    A = np.array([[1, p - 1], [2 % p, 1]], dtype=np.int32)
    for alpha, beta in itertools.product(range(p), range(p)):
        for c00, c10, c11, c01 in itertools.product(range(p), repeat=4):
            C = np.array([[c00, c01], [c10, c11]], dtype=np.int64)
            got = oracle.syrk_modp_low(alpha, A, beta, C, p).astype(np.int64)
            assert np.array_equal(got, _brute_syrk(alpha, A, beta, C, p))


def test_syrk_oracle_reduces_and_is_linear():
    p = 131071
    rng = np.random.default_rng(5)
    A = synth.residues(31, (9, 7), p)
    C = rng.integers(0, p, (9, 9))
    base = oracle.aat_modp_low(A, p).astype(np.int64)
    assert np.array_equal(oracle.syrk_modp_low(1, A, 0, C, p).astype(np.int64), base)
    assert np.array_equal(oracle.syrk_modp_low(0, A, 1, C, p).astype(np.int64), np.tril(C))
    a, b = 12345, 777
    got = oracle.syrk_modp_low(a, A, b, C, p).astype(np.int64)
    assert np.array_equal(got, np.tril((a * base + b * C) % p))
    # alpha = -1, beta = 1 on C = Low(A A^T): the zero matrix
    assert not oracle.syrk_modp_low(p - 1, A, 1, base, p).any()
    # all-ones A (k columns): alpha k + beta c_ij
    ones = np.ones((5, 11), dtype=np.int32)
    got = oracle.syrk_modp_low(3, ones, 2, np.full((5, 5), 4), p).astype(np.int64)
    assert np.array_equal(got, np.tril(np.full((5, 5), (3 * 11 + 2 * 4) % p)))


@pytest.mark.parametrize("p", [13, 17, 131071, 65521])
def test_syrk_table4_schedule_equals_definition(p):
    """The Table 4 schedule (one level of Algorithm 1, the locations the
    table names) gives Low(alpha A A^T + beta C), for Y of both kinds."""
    ykind, ya, yb = oracle.skew_unitary_params(p)
    # Table 4 holds for k <= n (S2 goes into C12)
    A = synth.residues(41, (8, 4 if ykind == 1 else 8), p)
    C = synth.residues(42, (8, 8), p).astype(np.int64)
    for alpha, beta in [(1, 0), (1, 1), (5, 3), (p - 1, 2)]:
        got = np.asarray(alg1.syrk_table4(alpha, A, beta, C, p, ykind, ya, yb), dtype=np.int64)
        want = oracle.syrk_modp_low(alpha, A, beta, C, p).astype(np.int64)
        assert np.array_equal(got, want), (alpha, beta)


def test_syrk_table4_literal_reading_loses_the_diagonal():
    """Taken literally, Up(C11) <- Low(C22)^T (Up includes the diagonal,
    Sec. 2) overwrites C11's diagonal before P2 = alpha A12 A12^T + beta C11
    reads it: the result is wrong whenever beta != 0 and the diagonals of
    C11 and C22 differ.  Hence the separate diagonal vector."""
    p = 131071
    ykind, ya, yb = oracle.skew_unitary_params(p)
    A = synth.residues(43, (8, 8), p)
    C = synth.residues(44, (8, 8), p).astype(np.int64)
    got = np.asarray(alg1.syrk_table4(1, A, 1, C, p, ykind, ya, yb, save_diagonal=False),
                     dtype=np.int64)
    want = oracle.syrk_modp_low(1, A, 1, C, p).astype(np.int64)
    # only the diagonal of the C11 block is lost
    assert not np.array_equal(np.diag(got)[:4], np.diag(want)[:4])
    assert np.array_equal(np.diag(got)[4:], np.diag(want)[4:])
    assert np.array_equal(np.tril(got, -1), np.tril(want, -1))


# ------------------------------------------------ quaternions (Sec. 6.2)

def _qmul(x, y, p):
    """Hamilton product of (a, b, c, d) = a + b i + c j + d k, mod p."""
    a1, b1, c1, d1 = x
    a2, b2, c2, d2 = y
    return ((a1 * a2 - b1 * b2 - c1 * c2 - d1 * d2) % p,
            (a1 * b2 + b1 * a2 + c1 * d2 - d1 * c2) % p,
            (a1 * c2 - b1 * d2 + c1 * a2 + d1 * b2) % p,
            (a1 * d2 + b1 * c2 - c1 * b2 + d1 * a2) % p)


def _brute_quat_aah(A, B, C, D, p):
    n, k = A.shape
    H = np.zeros((4, n, n), dtype=np.int64)
    for r in range(n):
        for c in range(n):
            acc = (0, 0, 0, 0)
            for l in range(k):
                x = (int(A[r, l]), int(B[r, l]), int(C[r, l]), int(D[r, l]))
                y = (int(A[c, l]), -int(B[c, l]), -int(C[c, l]), -int(D[c, l]))
                t = _qmul(x, y, p)
                acc = tuple((u + v) % p for u, v in zip(acc, t))
            H[:, r, c] = acc
    return H


def test_hamilton_units():
    """i^2 = j^2 = k^2 = ijk = -1, ij = k, ji = -k (the product used below)."""
    p = 101
    one, i, j, k = (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1)
    m1 = (p - 1, 0, 0, 0)
    assert _qmul(i, i, p) == m1 and _qmul(j, j, p) == m1 and _qmul(k, k, p) == m1
    assert _qmul(_qmul(i, j, p), k, p) == m1
    assert _qmul(i, j, p) == k and _qmul(j, i, p) == (0, 0, 0, p - 1)
    assert _qmul(one, j, p) == j


@pytest.mark.parametrize("p", [3, 7, 13, 131071])
def test_quat_oracle_against_hamilton_brute_force(p):
    n, k = 5, 4
    A, B, C, D = (synth.residues(70 + q, (n, k), p) for q in range(4))
    H = _brute_quat_aah(A, B, C, D, p)
    got = oracle.quat_aah_modp_low(A, B, C, D, p)
    for q in range(4):
        assert np.array_equal(got[q].astype(np.int64), np.tril(H[q]))
    # M M^H is quaternion-Hermitian: H1 symmetric, H2..H4 skew-symmetric
    assert np.array_equal(H[0], H[0].T)
    for q in (1, 2, 3):
        assert np.array_equal((H[q] + H[q].T) % p, np.zeros((n, n), dtype=np.int64))


def test_quat_oracle_special_cases():
    p = 65521
    A = synth.residues(81, (6, 9), p)
    Z = np.zeros_like(A)
    low = oracle.aat_modp_low(A, p).astype(np.int64)
    # a real matrix: H = A A^T, no imaginary parts
    got = oracle.quat_aah_modp_low(A, Z, Z, Z, p)
    assert np.array_equal(got[0].astype(np.int64), low) and not any(g.any() for g in got[1:])
    # A times a unit (i, j or k): (A u)(A u)^H = A A^T u conj(u) = A A^T
    for q in (1, 2, 3):
        parts = [Z, Z, Z, Z]
        parts[q] = A
        got = oracle.quat_aah_modp_low(*parts, p)
        assert np.array_equal(got[0].astype(np.int64), low) and not any(g.any() for g in got[1:])


@pytest.mark.parametrize("p", [5, 131071, 2**31 - 1])
def test_quat_6m_algorithm_equals_definition(p):
    """The 6-multiplication algorithm of Sec. 6.2 gives M M^H."""
    A, B, C, D = (synth.residues(90 + q, (7, 6), p) for q in range(4))
    want = oracle.quat_aah_modp_low(A, B, C, D, p)
    got = alg1.quat_6m(A, B, C, D, p)
    for q in range(4):
        assert np.array_equal(np.asarray(got[q], dtype=np.int64), want[q].astype(np.int64)), q


# --------------------------------------------- Winograd's form of Strassen

@pytest.mark.parametrize("p", [3, 13, 65521, 131071, 2**31 - 1])
@pytest.mark.parametrize("M,N,K", [(2, 2, 2), (4, 6, 8), (10, 4, 6), (12, 12, 20)])
def test_winograd_equals_definition(p, M, N, K):
    """One Winograd level equals the plain product X Y^T mod p."""
    X = synth.residues(p % 1000 + M * 7 + K, (M, K), p).astype(object)
    Y = synth.residues(p % 999 + N * 5 + K, (N, K), p).astype(object)
    ref = (X @ Y.T) % p
    tr = []
    got = alg1.winograd_gemm(X, Y, p, trace=tr)
    assert np.array_equal(got, ref)
    assert len(tr[0]["P"]) == 7            # seven block products
    # the C oracle's general product agrees as well
    assert np.array_equal(oracle.gemm_modp(X.astype(np.int64).astype(np.int32),
                                           Y.astype(np.int64).astype(np.int32), p)
                          .astype(np.int64).astype(object), ref)


def test_winograd_scalar_blocks_exhaustive_f3():
    """Every 2 x 2 X and Y over F_3 (1 x 1 blocks): 3^8 cases, brute force."""
    import itertools
    p = 3
    vals = list(itertools.product(range(3), repeat=4))
    for x in vals:
        X = np.array(x, dtype=object).reshape(2, 2)
        for y in vals:
            Y = np.array(y, dtype=object).reshape(2, 2)
            ref = np.array([[sum(X[i, l] * Y[j, l] for l in range(2)) % p for j in range(2)]
                            for i in range(2)], dtype=object)
            assert np.array_equal(alg1.winograd_gemm(X, Y, p), ref)


def test_winograd_every_product_contributes():
    """Dropping any one of the seven products changes the result: each
    block of C uses the products Winograd's form assigns to it."""
    p = 65521
    X = synth.residues(5, (4, 4), p).astype(object)
    Y = synth.residues(6, (4, 4), p).astype(object)
    tr = []
    alg1.winograd_gemm(X, Y, p, trace=tr)
    P = tr[0]["P"]
    uses = {0: {(0, 0), (0, 1), (1, 0), (1, 1)}, 1: {(0, 0)}, 2: {(0, 1)}, 3: {(1, 0)},
            4: {(0, 1), (1, 1)}, 5: {(0, 1), (1, 0), (1, 1)}, 6: {(1, 0), (1, 1)}}
    ref = (X @ Y.T) % p
    for q in range(7):
        assert np.any(P[q] % p != 0)
        # U1..U7 rebuilt without product q: the blocks that use it change
        Pz = [P[i] if i != q else 0 * P[i] for i in range(7)]
        U2 = Pz[0] + Pz[5]
        U3 = U2 + Pz[6]
        U4 = U2 + Pz[4]
        blocks = {(0, 0): Pz[0] + Pz[1], (0, 1): U4 + Pz[2], (1, 0): U3 - Pz[3],
                  (1, 1): U3 + Pz[4]}
        for (bi, bj), B in blocks.items():
            same = np.array_equal(B % p, ref[2 * bi:2 * bi + 2, 2 * bj:2 * bj + 2])
            assert same == ((bi, bj) not in uses[q])


@pytest.mark.parametrize("p", [65521, 131071, 2**31 - 1])
@pytest.mark.parametrize("n,k", [(8, 8), (16, 16), (16, 24)])
def test_alg1_with_winograd_general_products(p, n, k):
    """Algorithm 1 with Winograd's form for P3 and P4 gives the definition."""
    kind, a, b = oracle.skew_unitary_params(p)
    A = synth.residues(p % 1000 + 3 * n + k, (n, k), p)
    ref = _exact_low(A, p)
    for levels in (1, 2):
        if (n >> levels) % 2 or (k >> levels) % 2:
            continue
        C = alg1.alg1_low_aat(A, p, kind, a, b, levels, gemm=alg1.winograd_gemm)
        assert np.array_equal(C.astype(np.int64), ref), levels
