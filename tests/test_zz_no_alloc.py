"""aat_gemm_modp_noalloc: the allocation-free form of the general product.

It exists for callers that cannot allocate device memory when they call the
library (their host application owns all device memory, or an allocation on
the call path is not acceptable); its scratch lives in a fixed device array.
This file is collected last so that, if it fails, a run that stops at the
first failure has already run every other test.  It must pass on its own in
a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2101_01025_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_01025_gb300 import build
    build.build()
    from paper_2101_01025_gb300 import _native
    return _native


def _noalloc(nat, X, Y, p, C):
    stream = torch.cuda.current_stream().cuda_stream
    return nat.lib().aat_gemm_modp_noalloc(
        X.data_ptr(), X.stride(0), Y.data_ptr(), Y.stride(0), X.shape[0], Y.shape[0],
        X.shape[1], p, C.data_ptr(), C.stride(0), stream)


@pytest.mark.parametrize("p,m,n,k", [(2**31 - 1, 300, 520, 700), (65521, 257, 129, 1500),
                                     (131071, 1024, 1024, 1024)])
def test_noalloc_matches_allocating_entry_point_twice(lib, p, m, n, k):
    import paper_2101_01025_gb300 as aat
    X = torch.from_numpy(synth.residues(m + k, (m, k), p, balanced=True)).cuda()
    Y = torch.from_numpy(synth.residues(n + 3 * k, (n, k), p)).cuda()
    ref = aat.aat_gemm_modp(X, Y, p)          # the allocating entry point
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    for _ in range(2):                        # two calls in a row share the scratch
        C = torch.full((m, n), -1, dtype=torch.int32, device="cuda")
        lib.check(_noalloc(lib, X, Y, p, C))
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy(), ref)
    # X = Y (one set of planes)
    refs = aat.aat_gemm_modp(X, X, p).cpu().numpy()
    C = torch.full((m, m), -1, dtype=torch.int32, device="cuda")
    lib.check(_noalloc(lib, X, X, p, C))
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), refs)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    p = 2**31 - 1
    X = torch.zeros((2048, 2048), dtype=torch.int32, device="cuda")
    C = torch.zeros((2048, 2048), dtype=torch.int32, device="cuda")
    rc = _noalloc(lib, X, X, p, C)
    assert rc == lib.AAT_ERANGE
    assert "bytes of scratch" in lib.last_error()
