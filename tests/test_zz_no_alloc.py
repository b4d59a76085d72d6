"""grng_assign_static -- the nearest-pivot assignment that allocates nothing.

Some callers cannot allocate device memory (a pool that forbids new allocations, a
plugin whose host owns every allocation, a program whose footprint must stay fixed).
For them grng_assign_static does grng_build_layer's finest-layer assignment with all
scratch in a fixed array inside the library.  This test calls it through the C ABI and
checks it against grng_build_layer on two calls in a row (the second call runs on the
array the first one left behind).  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2208_10022_gb300 as g  # noqa: E402
from paper_2208_10022_gb300 import workloads as wl  # noqa: E402


def _static(X, piv, metric):
    L = g.lib()
    f = L.grng_assign_static
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                  ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    n, dim = X.shape
    assign = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    dist = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    st = f(X.data_ptr(), n, dim, piv.data_ptr(), piv.shape[0], metric, assign.data_ptr(), dist.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    return st, assign.cpu().numpy(), dist.cpu().numpy()


@pytest.mark.parametrize("kind,n,metric", [("lin96", 6000, wl.L2), ("mix16", 9000, wl.L1)])
def test_static_assignment_matches_build_layer(kind, n, metric):
    w = wl.make(kind, n=n, metric=metric)
    piv = w.layers[-1]
    ref = g.Index(w.X, n_layers=1, metric=metric)
    a_ref, r_ref, _ = ref.build_layer(0, piv)
    X = torch.from_numpy(w.X).cuda()
    P = torch.from_numpy(piv).cuda()
    for call in range(2):
        st, a, d = _static(X, P, metric)
        assert st == g.GRNG_OK, g.lib().grng_last_error()
        assert np.array_equal(a, a_ref), f"assignment differs on call {call}"
        r = np.zeros(len(piv))
        np.maximum.at(r, a, d)
        assert np.array_equal(r, r_ref), f"radii differ on call {call}"


def test_static_rejects_sizes_beyond_its_array():
    X = torch.zeros((300_000, 8), dtype=torch.float32, device="cuda")
    P = torch.arange(4, dtype=torch.int32, device="cuda")
    st, _, _ = _static(X, P, wl.L2)
    assert st == g.GRNG_EINVAL
    assert b"262144" in g.lib().grng_last_error()


def test_static_rejects_host_and_misaligned_buffers():
    """The call reads and writes the caller's buffers in place, so it checks on the host,
    before queueing any work, that each one is device memory on its access boundary."""
    n, dim = 512, 8
    P = torch.arange(4, dtype=torch.int32, device="cuda")
    Xh = np.zeros((n, dim), np.float32)                     # host memory
    L = g.lib()
    f = L.grng_assign_static
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                  ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    assign = torch.zeros(n, dtype=torch.int32, device="cuda")
    dist = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = f(Xh.ctypes.data, n, dim, P.data_ptr(), 4, wl.L2, assign.data_ptr(), dist.data_ptr(), None)
    assert st == g.GRNG_EINVAL and b"device" in L.grng_last_error()
    buf = torch.zeros(n * dim + 4, dtype=torch.float32, device="cuda")
    Xoff = buf[1:1 + n * dim].view(n, dim)                  # starts 4 bytes past a 16-byte boundary
    st = f(Xoff.data_ptr(), n, dim, P.data_ptr(), 4, wl.L2, assign.data_ptr(), dist.data_ptr(), None)
    assert st == g.GRNG_EINVAL and b"aligned" in L.grng_last_error()
    # the index buffers keep working afterwards
    X = buf[:n * dim].view(n, dim)
    st = f(X.data_ptr(), n, dim, P.data_ptr(), 4, wl.L2, assign.data_ptr(), dist.data_ptr(), None)
    assert st == g.GRNG_OK, L.grng_last_error()
