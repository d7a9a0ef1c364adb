"""Failure paths on the GPU without a GPU fault.

A bounded device wait that runs out: a probe kernel waits, with the bounded
mbarrier wait the leaf kernels use and a 2 ms limit, for a barrier phase that
nothing completes; the wait gives up, records AAT_ETIMEOUT in the status
word and the kernel returns.  aat_device_status must report it (for the
library's word and for the allocation-free entry point's own word), clear it
on request, and the library must keep working afterwards.  An allocation
that fails: the test allocation limit makes the workspace request of a
product fail with AAT_ENOMEM; C is left untouched and the next call, with
the limit lifted, is exact.
"""
import numpy as np
import pytest

import oracle
from paper_2101_01025_gb300 import _native, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_01025_gb300 import build
    build.build()
    import paper_2101_01025_gb300 as aat
    aat.aat_device_status(reset=True)
    yield aat
    assert aat.aat_device_status() == 0


def _small_product_is_exact(aat):
    p = 2**31 - 1
    A = synth.residues(77, (300, 200), p, balanced=True)
    C = aat.aat_modp(torch.from_numpy(A).cuda(), p)
    torch.cuda.synchronize()
    assert np.array_equal(np.tril(C.cpu().numpy().astype(np.int64)),
                          np.tril(oracle.aat_modp_low(A, p).astype(np.int64)))


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_times_out_and_reports(lib, which):
    nat = _native.lib()
    assert lib.aat_device_status() == 0
    stream = torch.cuda.current_stream().cuda_stream
    _native.check(nat.aatx_wait_probe(which, 2_000_000, stream))   # 2 ms
    assert lib.aat_device_status(reset=True) == _native.AAT_ETIMEOUT
    assert lib.aat_device_status() == 0      # cleared
    _small_product_is_exact(lib)             # the context is still usable
    assert lib.aat_device_status() == 0


def test_workspace_allocation_failure_gives_enomem(lib):
    nat = _native.lib()
    p = 2**31 - 1
    n = k = 1024
    A = torch.from_numpy(synth.residues(78, (n, k), p, balanced=True)).cuda()
    C = torch.full((n, n), -7, dtype=torch.int32, device="cuda")
    lib.aat_shutdown()                       # drop the workspace grown so far
    # below even the low-memory schedule's need (which the library falls back
    # to when the fast schedule's workspace cannot be allocated)
    need = lib.aat_workspace_size(n, k, p, lib.AAT_LOW_MEMORY)
    assert need > 0
    try:
        nat.aatx_set_alloc_limit(need // 2)
        with pytest.raises(lib.AatError) as ei:
            lib.aat_modp(A, p, C=C)
        assert ei.value.code == _native.AAT_ENOMEM
        torch.cuda.synchronize()
        assert int((C != -7).sum()) == 0     # nothing was launched
    finally:
        nat.aatx_set_alloc_limit(2**64 - 1)
    lib.aat_modp(A, p, C=C)
    torch.cuda.synchronize()
    ref = oracle.aat_modp_low(A.cpu().numpy(), p).astype(np.int64)
    assert np.array_equal(np.tril(C.cpu().numpy().astype(np.int64)), np.tril(ref))
