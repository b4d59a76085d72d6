"""Precision form: tensor-core (tcgen05, split BF16) distance tiles.

- the raw tile keys against FP64 keys, within the stated absolute bound, and far
  inside the error a single BF16 product would have (so both halves are in use);
- the exact RNG built on them: the edge set must equal the FP64 oracle's.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2208_10022_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2208_10022_gb300 as g  # noqa: E402


def _tc_keys(X):
    f = g.lib().grng_tc_keys
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    X = np.ascontiguousarray(X, np.float32)
    n, d = X.shape
    out = np.zeros((n, n), np.float32)
    st = f(X.ctypes.data, n, d, out.ctypes.data)
    assert st == g.GRNG_OK, g.lib().grng_last_error()
    return out


@pytest.mark.parametrize("n,d,scale", [(200, 96, 1.0), (256, 64, 10.0), (37, 16, 0.1), (130, 128, 1.0)])
def test_tc_tile_keys_within_bound(n, d, scale):
    rng = np.random.default_rng(n + d)
    X = (scale * rng.standard_normal((n, d))).astype(np.float32)
    got = _tc_keys(X).astype(np.float64)
    X64 = X.astype(np.float64)
    nrm = (X64 ** 2).sum(1)
    want = nrm[:, None] + nrm[None, :] - 2.0 * X64 @ X64.T
    Dp = ((d + 15) // 16) * 16
    gam = 2.0 ** -12 + (3 * Dp + 16) * 2.0 ** -24
    bound = gam * (nrm[:, None] + nrm[None, :])
    err = np.abs(got - want)
    assert np.all(err <= bound), float((err / bound).max())
    # a single BF16 product would be off by ~2^-8 |x||y|; the split keeps it far below
    assert np.median(err / (nrm[:, None] + nrm[None, :] + 1e-30)) < 2.0 ** -14


@pytest.mark.parametrize("n", [1500, 4000])
def test_bf16_build_equals_oracle(n):
    w = wl.make("lin96", n=n)
    ix, out = g.build_all(torch.from_numpy(w.X).cuda(), w.layers, metric=wl.L2, want_adjacency=False,
                          precision=g.BF16)
    got = {tuple(e) for e in out["edges"].tolist()}
    want = {tuple(e) for e in oracle.rng_brute(w.X).tolist()}
    assert got == want, len(got ^ want)
    st = ix.stats()
    assert st["rng"]["candidate_pairs"] > 0


def test_bf16_build_subsample_mixture():
    w = wl.make("mix16", n=100_000)
    s = wl.subsample(w, 6000, seed=3001)
    ix, out = g.build_all(s.X, s.layers, metric=wl.L2, precision=g.BF16)
    got = {tuple(e) for e in out["edges"].tolist()}
    want = {tuple(e) for e in oracle.rng_brute(s.X).tolist()}
    assert got == want, len(got ^ want)


def test_bf16_build_equals_fp32_build_many_tiles():
    # 20,000 points: 157 blocks, 24,649 tiles per sweep, a ragged last block; every tile of
    # the pipelined tensor-core sweep against the FP32 CUDA-core build (itself oracle-checked)
    w = wl.make("lin96", n=20000)
    _, o32 = g.build_all(w.X, w.layers, precision=g.FP32)
    ix, o16 = g.build_all(w.X, w.layers, precision=g.BF16)
    assert np.array_equal(o16["edges"], o32["edges"])
    st = ix.stats()["rng"]
    assert st["kernel_ms"]["tiles"] > 0


def test_bounded_wait_times_out_cleanly():
    """With a poll limit of one, the tensor-core sweep's first wait on a bulk copy runs out:
    the kernel drains what it issued, frees its tensor memory and reports GRNG_ETIMEOUT; the
    index can be destroyed and a new build on the same GPU gives the oracle's edges."""
    w = wl.make("lin96", n=3000)
    ix = g.Index(torch.from_numpy(w.X).cuda(), n_layers=len(w.layers), precision=g.BF16, spin_limit=1)
    for li in range(len(w.layers) - 1, -1, -1):
        ix.build_layer(li, w.layers[li], outputs=False)
    for li in range(len(w.layers)):
        ix.link_pivots(li, want_adjacency=False)
    with pytest.raises(g.GrngError) as e:
        ix.rng_build_exact()
    assert e.value.status == g.GRNG_ETIMEOUT
    ix.close()
    ix2, out = g.build_all(torch.from_numpy(w.X).cuda(), w.layers, precision=g.BF16)
    assert {tuple(e) for e in out["edges"].tolist()} == {tuple(e) for e in oracle.rng_brute(w.X).tolist()}
