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


@pytest.mark.parametrize("kind,n", [("lin96", 1500), ("lin96", 4000), ("lin128", 2500)])
def test_bf16_build_equals_oracle(kind, n):
    """lin96: the pipelined sweep (the next tile's copy and MMAs under this tile's
    epilogue); lin128: the form whose key tile reuses the operand buffer."""
    w = wl.make(kind, n=n)
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
    index can be destroyed and a new build on the same GPU gives the oracle's edges.  (One
    layer of 100 pivots: its assignment takes the FP32 tiles, below the tensor-core form's
    256 pivots, so the sweep is the first bounded wait.)"""
    w = wl.make("lin96", n=3000)
    layers = [np.sort(np.random.default_rng(4).choice(3000, 100, replace=False)).astype(np.int32)]
    ix = g.Index(torch.from_numpy(w.X).cuda(), n_layers=1, precision=g.BF16, spin_limit=1)
    ix.build_layer(0, layers[0], outputs=False)
    ix.link_pivots(0, want_adjacency=False)
    with pytest.raises(g.GrngError) as e:
        ix.rng_build_exact()
    assert e.value.status == g.GRNG_ETIMEOUT
    ix.close()
    ix2, out = g.build_all(torch.from_numpy(w.X).cuda(), layers, precision=g.BF16)
    assert {tuple(e) for e in out["edges"].tolist()} == {tuple(e) for e in oracle.rng_brute(w.X).tolist()}


def test_assignment_wait_times_out_cleanly():
    """The tensor-core assignment (a layer of at least 256 pivots) with a poll limit of one:
    GRNG_ETIMEOUT after its copies and MMAs are drained; the next index on the same GPU
    assigns exactly as the FP32 tiles do."""
    w = wl.make("lin96", n=6000)
    piv = w.layers[-1]
    assert len(piv) >= 256
    ix = g.Index(torch.from_numpy(w.X).cuda(), n_layers=1, precision=g.BF16, spin_limit=1)
    with pytest.raises(g.GrngError) as e:
        ix.build_layer(0, piv)
    assert e.value.status == g.GRNG_ETIMEOUT
    ix.close()
    a16, r16, _ = g.Index(w.X, n_layers=1, precision=g.BF16).build_layer(0, piv)
    a32, r32, _ = g.Index(w.X, n_layers=1, precision=g.FP32).build_layer(0, piv)
    assert np.array_equal(a16, a32) and np.array_equal(r16, r32)


@pytest.mark.parametrize("kind,n", [("lin96", 20000), ("mix16", 30000), ("lin128", 6000), ("ties16", 3000)])
def test_tc_assignment_equals_fp32(kind, n):
    """The nearest-pivot assignment from tensor-core Gram keys (the BF16 form) equals the
    FP32 one -- assignment, radii and delta_max bit for bit -- and the oracle's on a sample
    of members; members whose two nearest pivots the Gram bound cannot separate take the
    exact path (ties16: integer points with many exact ties)."""
    if kind == "ties16":
        rng = np.random.default_rng(31)
        X = rng.integers(0, 5, size=(n, 16)).astype(np.float32)
        piv = np.sort(rng.choice(n, 400, replace=False)).astype(np.int32)
    else:
        w = wl.make(kind, n=n)
        X, piv = w.X, w.layers[-1]
    a32, r32, d32 = g.Index(X, n_layers=1, precision=g.FP32).build_layer(0, piv)
    ix = g.Index(X, n_layers=1, precision=g.BF16)
    a16, r16, d16 = ix.build_layer(0, piv)
    assert np.array_equal(a32, a16), int((a32 != a16).sum())
    assert np.array_equal(r32, r16) and np.array_equal(d32, d16)
    rng = np.random.default_rng(32)
    sample = np.sort(rng.choice(X.shape[0], 200, replace=False)).astype(np.int32)
    oa = oracle.assign(X, sample, piv)[0]
    assert np.array_equal(oa, a16[sample])
    if kind == "ties16":
        assert ix.stats()["layers"][0]["assign_ambiguous"] > 0
