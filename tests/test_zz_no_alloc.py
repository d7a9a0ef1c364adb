"""aat_gemm_modp_noalloc: the allocation-free form of the general product.

It exists for callers that cannot allocate device memory when they call the
library (their host application owns all device memory, or an allocation on
the call path is not acceptable); its scratch lives in a fixed device array.
This file is collected last so that, if it fails, a run that stops at the
first failure has already run every other test.  It must pass on its own in
a fresh process as well as after the other tests.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2101_01025_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
def test_noalloc_matches_oracle_and_allocating_entry_point_twice(lib, p, m, n, k):
    import paper_2101_01025_gb300 as aat
    Xh = synth.residues(m + k, (m, k), p, balanced=True)
    Yh = synth.residues(n + 3 * k, (n, k), p)
    X = torch.from_numpy(Xh).cuda()
    Y = torch.from_numpy(Yh).cuda()
    want = oracle.gemm_modp(Xh, Yh, p).astype(np.int64)   # the definition
    ref = aat.aat_gemm_modp(X, Y, p)          # the allocating entry point
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    assert np.array_equal(ref.astype(np.int64), want)
    for _ in range(2):                        # two calls in a row share the scratch
        C = torch.full((m, n), -1, dtype=torch.int32, device="cuda")
        lib.check(_noalloc(lib, X, Y, p, C))
        torch.cuda.synchronize()
        got = C.cpu().numpy()
        assert np.array_equal(got, ref)
        assert np.array_equal(got.astype(np.int64), want)
    # X = Y (one set of planes)
    wants = oracle.gemm_modp(Xh, Xh, p).astype(np.int64)
    C = torch.full((m, m), -1, dtype=torch.int32, device="cuda")
    lib.check(_noalloc(lib, X, X, p, C))
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy().astype(np.int64), wants)
    assert np.array_equal(aat.aat_gemm_modp(X, X, p).cpu().numpy().astype(np.int64), wants)
    assert aat.aat_device_status() == 0       # both status words clear


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    p = 2**31 - 1
    X = torch.zeros((2048, 2048), dtype=torch.int32, device="cuda")
    C = torch.zeros((2048, 2048), dtype=torch.int32, device="cuda")
    rc = _noalloc(lib, X, X, p, C)
    assert rc == lib.AAT_ERANGE
    assert "bytes of scratch" in lib.last_error()


def test_noalloc_status_word_is_reported(lib):
    """A bounded wait that gives up on this entry point's own status word
    shows in aat_device_status (the probe waits 1 ms for a barrier phase that
    nothing completes; no fault)."""
    import paper_2101_01025_gb300 as aat
    assert aat.aat_device_status() == 0
    lib.check(lib.lib().aatx_wait_probe(1, 1_000_000, torch.cuda.current_stream().cuda_stream))
    assert aat.aat_device_status(reset=True) == lib.AAT_ETIMEOUT
    assert aat.aat_device_status() == 0


_CHILD = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import oracle
from paper_2101_01025_gb300 import _native, synth
torch.cuda.set_device(0)
p, m, n, k = 2**31 - 1, 1000, 1024, 1024
Xh = synth.residues(11, (m, k), p, balanced=True)
Yh = synth.residues(12, (n, k), p)
X, Y = torch.from_numpy(Xh).cuda(), torch.from_numpy(Yh).cuda()
C = torch.zeros((m, n), dtype=torch.int32, device="cuda")
tiny = torch.ones((1, 1), dtype=torch.int32, device="cuda")
st = torch.cuda.current_stream().cuda_stream
L = _native.lib()
def call(A, B, out):
    _native.check(L.aat_gemm_modp_noalloc(A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                  A.shape[0], B.shape[0], A.shape[1], p, out.data_ptr(), out.stride(0), st))
# first call on the device (a 1 x 1 product): loads the library's kernels and
# its static array, and looks the array's address up
t1 = torch.zeros((1, 1), dtype=torch.int32, device="cuda")
call(tiny, tiny, t1)
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
alloc0 = torch.cuda.memory_allocated()
for _ in range(2):
    call(X, Y, C)
    torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
assert torch.cuda.memory_allocated() == alloc0
assert abs(free1 - free0) <= (2 << 20), (free0, free1)
assert int(t1.item()) == 1
assert np.array_equal(C.cpu().numpy().astype(np.int64), oracle.gemm_modp(Xh, Yh, p).astype(np.int64))
print("free bytes before %d after %d" % (free0, free1))
"""


def test_noalloc_calls_leave_device_memory_unchanged(lib):
    """In a fresh process: after the first call on the device, two more calls
    (1000 x 1024 x 1024 over F_{2^31-1}) change neither the device's free
    memory (cudaMemGetInfo, within 2 MiB of driver-internal staging) nor
    torch's allocations, and the product equals the oracle's."""
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
