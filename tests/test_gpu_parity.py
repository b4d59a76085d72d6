"""GPU path against the FP64 oracle, element by element, through the C ABI.

Every case compares
  - each layer's assignment, radii and delta_max (bit-exact),
  - each layer's GRNG adjacency (exact edge sets),
  - the RNG edge list (exact edge set, sorted i < j),
with the oracle's definitions on the same seeded inputs.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2208_10022_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # collected on CPU machines, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2208_10022_gb300 as g  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "worked_examples.json")


def _edge_set(E):
    return {tuple(map(int, e)) for e in np.asarray(E).reshape(-1, 2)}


def _csr_rows(off, adj):
    return [set(adj[off[i]:off[i + 1]].tolist()) for i in range(len(off) - 1)]


def _rows_from_edges(E, m):
    rows = [set() for _ in range(m)]
    for i, j in np.asarray(E).reshape(-1, 2).tolist():
        rows[i].add(j)
        rows[j].add(i)
    return rows


def check_full(X, layers, metric, knn_k=32, on_gpu=True, flags=0):
    """Build everything on the GPU and compare every output with the oracle."""
    Xin = torch.from_numpy(X).cuda() if on_gpu else X
    ix, out = g.build_all(Xin, layers, metric=metric, knn_k=knn_k, want_adjacency=True, flags=flags)
    lay = oracle.build_layers(X, layers, metric)
    for li in range(len(layers)):
        a, r, dm = out["layers"][li]
        assert np.array_equal(a, lay[li]["assign"]), f"assignment of layer {li}"
        assert np.array_equal(r, lay[li]["radius"]), f"radii of layer {li}"
        assert np.array_equal(dm, lay[li]["delta_max"]), f"delta_max of layer {li}"
        off, adj = out["grng"][li]
        P = X[np.asarray(layers[li])]
        want = _rows_from_edges(oracle.grng_brute(P, lay[li]["radius"], metric), len(layers[li]))
        assert _csr_rows(off, adj) == want, f"GRNG of layer {li}"
    got = out["edges"]
    assert np.all(got[:, 0] < got[:, 1])
    assert np.array_equal(got, got[np.lexsort((got[:, 1], got[:, 0]))]), "edges not sorted"
    want = _edge_set(oracle.rng_brute(X, metric))
    assert _edge_set(got) == want, f"RNG: {len(_edge_set(got) ^ want)} edges differ"
    return ix


def test_worked_examples():
    gold = json.load(open(GOLDEN))
    for ex in gold["rng"]:
        X = np.asarray(ex["points"], np.float32)
        n = X.shape[0]
        layers = [np.array([0, n - 1], np.int32)] if n > 2 else [np.array([0], np.int32)]
        ix, out = g.build_all(X, layers, metric=ex["metric"])
        assert _edge_set(out["edges"]) == _edge_set(ex["edges"]), ex["name"]
    for ex in gold["grng"]:
        P = np.asarray(ex["points"], np.float32)
        m = P.shape[0]
        ix = g.Index(P, n_layers=1, metric=ex["metric"])
        ix.build_layer(0, np.arange(m, dtype=np.int32))
        off, adj = ix.link_pivots(0, radius_override=np.asarray(ex["radii"], np.float64))
        assert _csr_rows(off, adj) == _rows_from_edges(ex["edges"], m), ex["name"]


@pytest.mark.parametrize("metric", [wl.L2, wl.L1])
def test_plain_uniform8(metric):
    """1,000 points in [0,1]^8, one layer of 32 random pivots (the plain configuration)."""
    w = wl.make("uniform8", metric=metric)
    check_full(w.X, w.layers, metric)


@pytest.mark.parametrize("metric", [wl.L2, wl.L1])
def test_mixture_two_layers(metric):
    w = wl.make("mix16", n=3000, metric=metric)
    check_full(w.X, w.layers, metric)


def test_linear_manifold_three_layers():
    w = wl.make("lin96", n=2500)
    check_full(w.X, w.layers, wl.L2)


def test_ragged_sizes_and_odd_dims():
    rng = np.random.default_rng(5)
    for n, d in [(1, 3), (2, 1), (3, 5), (129, 17), (300, 33), (257, 2)]:
        X = rng.standard_normal((n, d)).astype(np.float32)
        m = max(1, n // 9)
        fine = np.sort(rng.choice(n, size=m, replace=False)).astype(np.int32)
        for metric in (wl.L2, wl.L1):
            if n >= 2:
                check_full(X, [fine], metric, on_gpu=False)


def test_ties_and_duplicates():
    rng = np.random.default_rng(6)
    X = rng.integers(0, 4, size=(300, 2)).astype(np.float32)   # many duplicates and exact ties
    for metric in (wl.L2, wl.L1):
        fine = np.sort(rng.choice(300, size=40, replace=False)).astype(np.int32)
        coarse = np.sort(rng.choice(fine, size=6, replace=False)).astype(np.int32)
        check_full(X, [coarse, fine], metric)


def test_small_knn_lists():
    """Short neighbour lists push many pairs into the hierarchical exhaustive tier."""
    w = wl.make("mix16", n=1500)
    for k in (1, 4):
        check_full(w.X, w.layers, wl.L2, knn_k=k)
    w = wl.make("lin96", n=2500)
    ix = check_full(w.X, w.layers, wl.L2, knn_k=1)
    st = ix.stats()
    assert st["rng"]["tier3_pairs"] > 0 and st["layers"][2]["grng"]["range_pairs"] > 0
    # capped range lists: the hierarchical exhaustive tier takes the pivot pairs
    ix = check_full(w.X, w.layers, wl.L2, knn_k=1, flags=g.GRNG_FLAG_SHORT_LISTS)
    st = ix.stats()
    assert st["layers"][2]["grng"]["range_lists_cut"] > 0 and st["layers"][2]["grng"]["tier3_pairs"] > 0
    check_full(w.X, w.layers, wl.L1, knn_k=2, flags=g.GRNG_FLAG_SHORT_LISTS)


def test_zero_radius_override_is_rng_of_pivots():
    w = wl.make("uniform8", n=800, layer_sizes=[200])
    ix = g.Index(w.X, n_layers=1)
    ix.build_layer(0, w.layers[0])
    off, adj = ix.link_pivots(0, radius_override=np.zeros(200))
    P = w.X[w.layers[0]]
    assert _csr_rows(off, adj) == _rows_from_edges(oracle.rng_brute(P), 200)


@pytest.mark.parametrize("metric", [wl.L2, wl.L1])
def test_subsample_10k_mixture(metric):
    """The seeded 10,000-point subsample of the 100,000-point mixture, pivots scaled x0.1."""
    w = wl.make("mix16", metric=metric)
    s = wl.subsample(w, 10_000, seed=3001)
    check_full(s.X, s.layers, metric)


def test_api_errors():
    X = np.zeros((10, 3), np.float32)
    with pytest.raises(g.GrngError) as e:
        g.Index(X, n_layers=0)
    assert e.value.status == g.GRNG_EINVAL
    ix = g.Index(X, n_layers=2)
    with pytest.raises(g.GrngError) as e:
        ix.build_layer(0, np.array([1, 2], np.int32))   # finer layer not built yet
    assert e.value.status == g.GRNG_ESTATE
    with pytest.raises(g.GrngError) as e:
        ix.build_layer(1, np.array([1, 1], np.int32))   # duplicate pivot
    assert e.value.status == g.GRNG_EINVAL
    ix.build_layer(1, np.array([1, 2, 3], np.int32))
    with pytest.raises(g.GrngError) as e:
        ix.build_layer(0, np.array([4], np.int32))      # not nested
    assert e.value.status == g.GRNG_EINVAL
    with pytest.raises(g.GrngError) as e:
        ix.rng_build_exact()
    assert e.value.status == g.GRNG_ESTATE


def test_small_buffers_take_every_overflow_path():
    """With every internal buffer started tiny, the tier-1 sweep and tiers 2-3 repeat with
    larger buffers and the exhaustive tier falls back to scanning every node; the graphs
    stay the oracle's."""
    w = wl.make("lin96", n=2500)
    flags = g.GRNG_FLAG_SMALL_BUFFERS | g.GRNG_FLAG_SHORT_LISTS
    ix = check_full(w.X, w.layers, wl.L2, knn_k=1, flags=flags)
    st = ix.stats()
    levels = [L["grng"] for L in st["layers"]] + [st["rng"]]
    assert max(L["tier1_attempts"] for L in levels) >= 2
    assert sum(L["tier3_overflows"] for L in levels) > 0
    rng = np.random.default_rng(6)
    X = rng.integers(0, 4, size=(300, 2)).astype(np.float32)   # exact ties: many FP64 rechecks
    fine = np.sort(rng.choice(300, size=40, replace=False)).astype(np.int32)
    coarse = np.sort(rng.choice(fine, size=6, replace=False)).astype(np.int32)
    ix = check_full(X, [coarse, fine], wl.L2, knn_k=1, flags=flags)
    st = ix.stats()
    levels = [L["grng"] for L in st["layers"]] + [st["rng"]]
    assert max(L["tier23_attempts"] for L in levels) >= 2
    w = wl.make("mix16", n=3000, metric=wl.L1)
    check_full(w.X, w.layers, wl.L1, knn_k=2, flags=flags)


def test_small_buffers_tensor_core_sweep():
    """The tensor-core exemplar sweep repeats with a larger survivor buffer."""
    w = wl.make("lin96", n=3000)
    ix, out = g.build_all(torch.from_numpy(w.X).cuda(), w.layers, precision=g.BF16, knn_k=4,
                          flags=g.GRNG_FLAG_SMALL_BUFFERS)
    assert _edge_set(out["edges"]) == _edge_set(oracle.rng_brute(w.X))
    assert ix.stats()["rng"]["tier1_attempts"] >= 2


def test_range_lists_intersect_and_scan():
    """Pivot pairs decided from range lists, covered from one side and from both; the
    layer's GRNG stays the oracle's."""
    w = wl.make("lin96", n=6000)
    ix = check_full(w.X, w.layers, wl.L2, knn_k=1)
    G = ix.stats()["layers"][-1]["grng"]
    assert G["range_pairs"] > 0 and G["range_both_covered"] > 0 and G["range_nodes_tested"] > 0, G
