"""Batched plans (aat_plan_*): many independent products in one graph launch.

Every F_p result is compared bit for bit with the oracle (in full for small
problems, sampled entries + Freivalds for large ones); complex results by
relative Frobenius error.  A plan is executed twice with the inputs changed
in between: the second execution must reflect the new inputs.
"""
import numpy as np
import pytest

import oracle
from paper_2101_01025_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def _fp_check(A, C, p, full):
    n = A.shape[0]
    if full:
        ref = oracle.aat_modp_low(A, p).astype(np.int64)
        assert np.array_equal(np.tril(C.astype(np.int64)), ref)
        return
    rng = np.random.default_rng(n)
    i = rng.integers(0, n, 400)
    j = rng.integers(0, n, 400)
    ij = np.stack([np.maximum(i, j), np.minimum(i, j)], 1)
    ij = np.concatenate([ij, [[n - 1, 0], [n - 1, n - 1], [0, 0]]])
    ref = oracle.aat_modp_entries(A, p, ij).astype(np.int64)
    assert np.array_equal(C[ij[:, 0], ij[:, 1]].astype(np.int64), ref)
    assert oracle.freivalds_modp(A, C, p, synth.vectors_mod_p(n, 1, n, p)) == 0


def test_plan_mixed_batch_twice(lib):
    rng_n = synth.log_uniform_ints(11, 30, 40, 700)
    rng_k = synth.log_uniform_ints(12, 30, 40, 900)
    problems, hosts = [], []
    primes = [65521, 131071, 2**31 - 1, 13]
    for q, (n, k) in enumerate(zip(rng_n, rng_k)):
        p = primes[q % 4]
        A = synth.residues(100 + q, (n, k), p)
        Ad = torch.from_numpy(A).cuda()
        Cd = torch.full((n, n), -1, dtype=torch.int32, device="cuda")
        problems.append(("modp", Ad, Cd, p, 0))
        hosts.append(("modp", A, Ad, Cd, p))
    # a recursive product (runs on its own) and complex products
    A = synth.residues(7, (520, 640), 2**31 - 1)
    Ad, Cd = torch.from_numpy(A).cuda(), torch.zeros((520, 520), dtype=torch.int32, device="cuda")
    problems.append(("modp", Ad, Cd, 2**31 - 1, lib.AAT_LEVELS(1)))
    hosts.append(("modp", A, Ad, Cd, 2**31 - 1))
    for q, kind in enumerate(["aah", "aat_c", "aah"]):
        n, k = 300 + 37 * q, 200 + 51 * q
        Z = synth.complex_normal(50 + q, (n, k))
        Zd = torch.from_numpy(Z).cuda()
        Cz = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
        problems.append((kind, Zd, Cz, 0, 0))
        hosts.append((kind, Z, Zd, Cz, None))
    plan = lib.Plan(problems)
    info = plan.info()
    # 30 depth-0 F_p problems and the two A A^H ones are batched; the
    # recursive product and the complex A A^T run on their own
    assert info["batched"] == 32 and info["solo"] == 2
    for rnd in range(2):
        if rnd == 1:   # new inputs: the plan must read them
            for idx, (kind, A, Ad, Cd, p) in enumerate(hosts):
                if kind == "modp":
                    A2 = synth.residues(900 + idx, A.shape, p)
                    Ad.copy_(torch.from_numpy(A2))
                    hosts[idx] = (kind, A2, Ad, Cd, p)
        plan.execute()
        torch.cuda.synchronize()
        for kind, A, Ad, Cd, p in hosts:
            C = Cd.cpu().numpy()
            if kind == "modp":
                _fp_check(A, C, p, full=True)
            else:
                ref = oracle.complex_low(A.astype(np.complex128), conj=(kind == "aah"))
                err = np.linalg.norm(np.tril(C - ref)) / np.linalg.norm(np.tril(ref))
                assert err <= 1e-5, (kind, err)
    plan.close()


def test_plan_rejects_bad_problems(lib):
    Ad = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(lib.AatError):
        lib.Plan([("modp", Ad, Ad.clone(), 15, 0)])     # 15 is not prime


def test_plan_config5_batch(lib):
    """256 F_p problems, p = 65521, n log-uniform in [64, 2048], k in
    [64, 4096], plus 64 complex FP32 problems of the same spread."""
    p = 65521
    ns = synth.log_uniform_ints(synth.SEED_BASE + 4, 256, 64, 2048)
    ks = synth.log_uniform_ints(synth.SEED_BASE + 5, 256, 64, 4096)
    problems, hosts = [], []
    for q in range(256):
        A = synth.residues(synth.SEED_BASE + 1000 + q, (ns[q], ks[q]), p)
        Ad = torch.from_numpy(A).cuda()
        Cd = torch.empty((ns[q], ns[q]), dtype=torch.int32, device="cuda")
        problems.append(("modp", Ad, Cd, p, 0))
        hosts.append((A, Cd))
    cn = synth.log_uniform_ints(synth.SEED_BASE + 6, 64, 64, 2048)
    ck = synth.log_uniform_ints(synth.SEED_BASE + 7, 64, 64, 4096)
    chosts = []
    for q in range(64):
        Z = synth.complex_normal(synth.SEED_BASE + 2000 + q, (cn[q], ck[q]))
        Zd = torch.from_numpy(Z).cuda()
        Cz = torch.empty((cn[q], cn[q]), dtype=torch.complex64, device="cuda")
        problems.append(("aah", Zd, Cz, 0, 0))
        chosts.append((Z, Cz))
    plan = lib.Plan(problems)
    plan.execute()
    torch.cuda.synchronize()
    for A, Cd in hosts:
        _fp_check(A, Cd.cpu().numpy(), p, full=A.shape[0] * A.shape[0] * A.shape[1] < 2e8)
    rng = np.random.default_rng(3)
    for Z, Cz in chosts:
        n = Z.shape[0]
        i = rng.integers(0, n, 200)
        j = rng.integers(0, n, 200)
        d = rng.integers(0, n, 20)   # diagonal entries (the FP64 sums)
        ij = np.concatenate([np.stack([np.maximum(i, j), np.minimum(i, j)], 1),
                             np.stack([d, d], 1)])
        ref = oracle.complex_entries(Z.astype(np.complex128), ij, conj=True)
        got = Cz.cpu().numpy()[ij[:, 0], ij[:, 1]]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    plan.close()


@pytest.mark.parametrize("flags", [1 << 16, 2 << 16])
def test_plan_complex_batch_precisions(lib, flags):
    """The batched complex path with 2 and 1 BF16 pieces per value, ragged
    sizes, against the FP64 oracle (the tolerances of the single calls)."""
    problems, hosts = [], []
    for q, (n, k) in enumerate([(33, 70), (300, 257), (129, 1000), (700, 64)]):
        Z = synth.complex_normal(300 + q, (n, k))
        Zd = torch.from_numpy(Z).cuda()
        Cz = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
        problems.append(("aah", Zd, Cz, 0, flags))
        hosts.append((Z, Cz))
    plan = lib.Plan(problems)
    assert plan.info()["batched"] == 4 and plan.info()["solo"] == 0
    plan.execute()
    torch.cuda.synchronize()
    # plain BF16: the bound of the single calls, also for n >> k (700 x 64),
    # where the exact FP64 diagonal carries little of the norm
    tol = 1e-4 if flags == 1 << 16 else 3e-3
    for Z, Cz in hosts:
        ref = oracle.complex_low(Z.astype(np.complex128), conj=True)
        C = Cz.cpu().numpy()
        err = np.linalg.norm(np.tril(C - ref)) / np.linalg.norm(np.tril(ref))
        assert err <= tol, err
        assert np.all(np.abs(np.diag(C).imag) == 0) and np.all(np.diag(C).real >= 0)
    plan.close()


def test_plan_with_low_memory_problems(lib):
    """Recursive products on the low-memory schedule (S blocks in C, plane
    passes) inside a plan's graph, run twice with new inputs."""
    problems, hosts = [], []
    for q, (n, k, p, lv) in enumerate([(1024, 768, 2**31 - 1, 1), (1024, 1024, 65521, 2),
                                       (776, 520, 2**31 - 1, 2)]):
        A = synth.residues(400 + q, (n, k), p)
        Ad = torch.from_numpy(A).cuda()
        Cd = torch.full((n, n), -1, dtype=torch.int32, device="cuda")
        problems.append(("modp", Ad, Cd, p, lib.AAT_LEVELS(lv) | lib.AAT_LOW_MEMORY))
        hosts.append((A, Ad, Cd, p))
    plan = lib.Plan(problems)
    assert plan.info()["solo"] == 3
    for rnd in range(2):
        if rnd == 1:
            for idx, (A, Ad, Cd, p) in enumerate(hosts):
                A2 = synth.residues(800 + idx, A.shape, p)
                Ad.copy_(torch.from_numpy(A2))
                hosts[idx] = (A2, Ad, Cd, p)
        plan.execute()
        torch.cuda.synchronize()
        for A, Ad, Cd, p in hosts:
            _fp_check(A, Cd.cpu().numpy(), p, full=True)
    plan.close()


def test_plan_with_winograd_problems(lib):
    """Recursive products with Winograd's form for their last level's
    general products, captured in the plan's graph and run twice."""
    problems, hosts = [], []
    for q, (n, k, p, lv) in enumerate([(1024, 768, 2**31 - 1, 1), (1024, 1024, 65521, 2),
                                       (776, 520, 131071, 1)]):
        A = synth.residues(300 + q, (n, k), p)
        Ad = torch.from_numpy(A).cuda()
        Cd = torch.full((n, n), -1, dtype=torch.int32, device="cuda")
        problems.append(("modp", Ad, Cd, p, lib.AAT_LEVELS(lv) | lib.AAT_WINOGRAD))
        hosts.append((A, Ad, Cd, p))
    plan = lib.Plan(problems)
    assert plan.info()["solo"] == 3
    for rnd in range(2):
        if rnd == 1:
            for idx, (A, Ad, Cd, p) in enumerate(hosts):
                A2 = synth.residues(700 + idx, A.shape, p)
                Ad.copy_(torch.from_numpy(A2))
                hosts[idx] = (A2, Ad, Cd, p)
        plan.execute()
        torch.cuda.synchronize()
        for A, Ad, Cd, p in hosts:
            _fp_check(A, Cd.cpu().numpy(), p, full=True)
    plan.close()


def test_plan_long_k_tiles_with_many_groups(lib):
    """Batched depth-0 products over F_{2^31-1} whose K spans several 8192-wide
    segments: 10 plane products per segment make 51 and 61 groups per tile,
    more than the 32 the batched epilogue keeps in shared memory, so the
    later groups come from global memory on every role of the kernel."""
    p = 2**31 - 1
    shapes = [(96, 41000), (130, 33000), (200, 300)]
    problems, hosts = [], []
    for q, (n, k) in enumerate(shapes):
        A = synth.residues(700 + q, (n, k), p, balanced=(q % 2 == 0))
        Ad = torch.from_numpy(A).cuda()
        Cd = torch.full((n, n), -1, dtype=torch.int32, device="cuda")
        problems.append(("modp", Ad, Cd, p, 0))
        hosts.append((A, Cd))
    plan = lib.Plan(problems)
    assert plan.info()["batched"] == 3
    plan.execute()
    torch.cuda.synchronize()
    for A, Cd in hosts:
        _fp_check(A, Cd.cpu().numpy(), p, full=True)
    plan.close()
