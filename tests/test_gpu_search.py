"""RNG search (rng_search_batch, Algorithm 1 without Stage VII) through the C ABI: each
query's neighbours among the index points equal the FP64 oracle's (Eq. 1 over the index
plus that query alone), element by element.  Queries come from the same generator as the
index, plus duplicates of index points and of pivots, and far points that lie in no
pivot's ball (no Theorem 1 filter for them).  The index is left unchanged."""
import numpy as np
import pytest

import oracle
from paper_2208_10022_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # collected on CPU machines, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2208_10022_gb300 as g  # noqa: E402


def _es(E):
    return {tuple(e) for e in np.asarray(E).reshape(-1, 2).tolist()}


def _queries(w, extra, seed):
    """`extra` fresh points of the same generator, then duplicates of two index points and
    of a fine pivot, then two far points (scaled by 20 about the mean)."""
    kind = w.name.split("-")[0]
    fresh = wl.gen_points(kind, w.n + extra, wl.SPECS[kind][3])[w.n:]
    rng = np.random.default_rng(seed)
    dup = w.X[rng.choice(w.n, 2, replace=False)]
    piv = w.X[w.layers[-1][:1]]
    mu = w.X.mean(0)
    far = (mu + 20.0 * (w.X[rng.choice(w.n, 2, replace=False)] - mu)).astype(np.float32)
    return np.ascontiguousarray(np.concatenate([fresh, dup, piv, far]).astype(np.float32))


def _check(ix, X, Q, metric):
    got = ix.rng_search(Q)
    want = oracle.rng_search(X, Q.cpu().numpy() if torch.is_tensor(Q) else Q, metric)
    bad = [j for j in range(len(Q)) if not np.array_equal(got[j], want[j])]
    assert not bad, f"{len(bad)} of {len(Q)} queries differ, e.g. query {bad[0]}: {got[bad[0]]} vs {want[bad[0]]}"
    return got


@pytest.mark.parametrize("kind,n,metric,precision", [
    ("mix16", 4000, wl.L2, g.FP32),
    ("uniform8", 3000, wl.L1, g.FP32),
    ("lin96", 3000, wl.L2, g.BF16),
])
def test_search_matches_oracle(kind, n, metric, precision):
    w = wl.make(kind, n=n, metric=metric)
    Q = _queries(w, 295, seed=21)                 # 300 queries: three strips, the last ragged
    ix, out = g.build_all(w.X, w.layers, metric=metric, precision=precision)
    E0 = out["edges"].copy()
    got = _check(ix, w.X, Q, metric)
    assert all(len(r) >= 1 for r in got)          # the nearest index point is always a neighbour
    dup_ids = np.flatnonzero((w.X == Q[295]).all(1))
    assert set(dup_ids.tolist()) <= set(got[295].tolist())  # a duplicate is linked
    assert _es(ix.rng_edges()) == _es(E0)        # the index is unchanged
    st = ix.stats()["search"]
    assert st["batches"] == 1 and st["queries"] == len(Q)
    assert st["outside_ball"] >= 2                # the far points: no pivot ball holds them
    assert st["neighbours"] == sum(len(r) for r in got)


def test_search_sizes_and_reuse():
    """One query, then a batch larger than the cached rows, then a small one again, on a
    three-layer lin96 index (K = 8); results through device buffers as well."""
    w = wl.make("lin96", n=2500)
    ix, _ = g.build_all(torch.from_numpy(w.X).cuda(), w.layers, knn_k=8)
    Q = _queries(w, 700, seed=22)
    _check(ix, w.X, Q[:1], wl.L2)
    _check(ix, w.X, torch.from_numpy(Q).cuda(), wl.L2)
    _check(ix, w.X, Q[-5:], wl.L2)
    total = ix.rng_search_batch(torch.from_numpy(Q[:40]).cuda())
    off = torch.zeros(41, dtype=torch.int64, device="cuda")
    nb = torch.zeros(total, dtype=torch.int32, device="cuda")
    off, nb = ix.rng_search_result(off, nb)
    want = oracle.rng_search(w.X, Q[:40])
    off = off.cpu().numpy()
    nb = nb.cpu().numpy()
    assert int(off[-1]) == total
    for j in range(40):
        assert np.array_equal(nb[off[j]:off[j + 1]], want[j])


def test_search_after_insertion():
    """A search after a batched insertion sees the inserted points."""
    full = wl.make("mix16", n=3000)
    n0 = 2400
    rng = np.random.default_rng(6)
    fine = np.sort(rng.choice(n0, 80, replace=False)).astype(np.int32)
    coarse = np.sort(rng.choice(fine, 10, replace=False)).astype(np.int32)
    ix, _ = g.build_all(full.X[:n0], [coarse, fine])
    Q = wl.gen_points("mix16", 3100, 77)[3000:]
    _check(ix, full.X[:n0], Q, wl.L2)
    ix.rng_insert_batch(full.X[n0:])
    _check(ix, full.X, Q, wl.L2)
    assert _es(ix.rng_edges()) == _es(oracle.rng_brute(full.X))


@pytest.mark.parametrize("metric", [wl.L2, wl.L1])
def test_search_integer_ties(metric):
    """Small integer coordinates: many exactly equal keys, duplicates in the index and
    among the queries; the small-buffers mode runs every retry path."""
    rng = np.random.default_rng(23)
    X = rng.integers(0, 6, size=(900, 4)).astype(np.float32)
    Q = np.concatenate([rng.integers(0, 6, size=(150, 4)), X[:10]]).astype(np.float32)
    rng2 = np.random.default_rng(24)
    fine = np.sort(rng2.choice(900, 40, replace=False)).astype(np.int32)
    coarse = np.sort(rng2.choice(fine, 6, replace=False)).astype(np.int32)
    ix, _ = g.build_all(X, [coarse, fine], metric=metric, flags=g.GRNG_FLAG_SMALL_BUFFERS)
    _check(ix, X, Q, metric)


def test_search_errors():
    """Invalid calls fail on the host with a status, before any device work."""
    w = wl.make("uniform8", n=500)
    ix = g.Index(w.X, n_layers=1)
    with pytest.raises(g.GrngError) as e:
        ix.rng_search_result()
    assert e.value.status in (g.GRNG_ESTATE,)
    ix.build_layer(0, w.layers[-1])
    with pytest.raises(g.GrngError) as e:
        ix.rng_search_batch(w.X[:3])                # the layer is not linked
    assert e.value.status == g.GRNG_ESTATE
    ix.link_pivots(0, want_adjacency=False)
    with pytest.raises(g.GrngError) as e:
        ix.rng_search_batch(np.zeros((0, 8), np.float32))
    assert e.value.status == g.GRNG_EINVAL
    total = ix.rng_search_batch(w.X[:4] + 0.01)
    off = np.zeros(5, np.int64)
    nb = np.zeros(max(total - 1, 1), np.int32)
    st = g.lib().rng_search_result(ix._h, off.ctypes.data, nb.ctypes.data, total - 1)
    assert st == g.GRNG_ETRUNC and off[-1] == total
