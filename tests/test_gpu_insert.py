"""Batched insertion (rng_insert_batch) through the C ABI: after each batch of uneven size
the stored RNG equals the FP64 oracle's RNG of all points so far, and a from-scratch
build on the enlarged set with the same pivots gives the same edges and GRNGs.  The
insertion is incremental (Algorithm 1, Stage VII): the statistics show the batch rows'
candidate pairs, the pivot pairs re-tested after radii grew and the old edges removed."""
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


@pytest.mark.parametrize("kind,metric", [("mix16", wl.L2), ("uniform8", wl.L1)])
def test_batches_match_oracle_and_rebuild(kind, metric):
    full = wl.make(kind, n=3600, metric=metric)
    sizes = [1, 317, 1000, 82]
    n0 = full.n - sum(sizes)
    # pivots drawn among the first n0 points (the points present at the first build)
    rng = np.random.default_rng(5)
    fine = np.sort(rng.choice(n0, 96, replace=False)).astype(np.int32)
    coarse = np.sort(rng.choice(fine, 12, replace=False)).astype(np.int32)
    layers = [coarse, fine]
    ix, out = g.build_all(full.X[:n0], layers, metric=metric)
    assert _es(out["edges"]) == _es(oracle.rng_brute(full.X[:n0], metric))
    at = n0
    for b in sizes:
        ix.rng_insert_batch(full.X[at:at + b])
        at += b
        got = _es(ix.rng_edges())
        assert got == _es(oracle.rng_brute(full.X[:at], metric)), f"after {at} points"
    st = ix.stats()
    assert st["insert"]["batches"] == len(sizes) and st["insert"]["points"] == sum(sizes)
    ix2, out2 = g.build_all(full.X[:at], layers, metric=metric, want_adjacency=True)
    assert _es(out2["edges"]) == got
    for li in range(2):
        off, adj = ix.adjacency_rows(li, 0, len(layers[li]))
        off2, adj2 = out2["grng"][li]
        assert np.array_equal(off, off2) and np.array_equal(adj, adj2), f"GRNG of layer {li}"


def _check_against_rebuild(ix, X, layers, metric):
    ix2, out2 = g.build_all(X, layers, metric=metric, want_adjacency=True)
    assert _es(out2["edges"]) == _es(ix.rng_edges())
    for li in range(len(layers)):
        off, adj = ix.adjacency_rows(li, 0, len(layers[li]))
        off2, adj2 = out2["grng"][li]
        assert np.array_equal(off, off2) and np.array_equal(adj, adj2), f"GRNG of layer {li}"


@pytest.mark.parametrize("flags", [0, g.GRNG_FLAG_SMALL_BUFFERS])
def test_three_layers_incremental(flags):
    """lin96 with three pivot layers, five batches (one of a single point); every batch is
    checked against the oracle, the last state against a rebuild."""
    full = wl.make("lin96", n=3000)
    sizes = [400, 1, 57, 640, 233]
    n0 = full.n - sum(sizes)
    rng = np.random.default_rng(8)
    fine = np.sort(rng.choice(n0, 160, replace=False)).astype(np.int32)
    mid = np.sort(rng.choice(fine, 40, replace=False)).astype(np.int32)
    top = np.sort(rng.choice(mid, 6, replace=False)).astype(np.int32)
    layers = [top, mid, fine]
    ix, _ = g.build_all(torch.from_numpy(full.X[:n0]).cuda(), layers, knn_k=8, flags=flags)
    at = n0
    for b in sizes:
        ix.rng_insert_batch(torch.from_numpy(full.X[at:at + b]).cuda())
        at += b
        assert _es(ix.rng_edges()) == _es(oracle.rng_brute(full.X[:at])), f"after {at} points"
    ins = ix.stats()["insert"]
    assert ins["batches"] == len(sizes) and ins["points"] == sum(sizes)
    assert ins["candidate_pairs"] > 0 and ins["new_edges"] > 0
    assert ins["removed_edges"] > 0 and ins["changed_pivots"] > 0
    _check_against_rebuild(ix, full.X[:at], layers, wl.L2)


def test_insert_duplicates_and_ties():
    """Integer points with many exact ties; the batch repeats existing points (a duplicate
    is always linked to its twin and never blocks, Eq. 1 read literally)."""
    rng = np.random.default_rng(9)
    X = rng.integers(0, 5, size=(260, 2)).astype(np.float32)
    B = np.concatenate([X[:20], rng.integers(0, 5, size=(30, 2)).astype(np.float32)])
    fine = np.sort(rng.choice(260, 30, replace=False)).astype(np.int32)
    coarse = np.sort(rng.choice(fine, 5, replace=False)).astype(np.int32)
    for metric in (wl.L2, wl.L1):
        ix, _ = g.build_all(X, [coarse, fine], metric=metric)
        ix.rng_insert_batch(B[:7])
        ix.rng_insert_batch(B[7:])
        XA = np.concatenate([X, B])
        assert _es(ix.rng_edges()) == _es(oracle.rng_brute(XA, metric))
        _check_against_rebuild(ix, XA, [coarse, fine], metric)


def test_insert_errors():
    w = wl.make("uniform8", n=300)
    ix = g.Index(w.X, n_layers=1)
    with pytest.raises(g.GrngError) as e:
        ix.rng_insert_batch(w.X[:5])
    assert e.value.status == g.GRNG_ESTATE
    ix.build_layer(0, w.layers[-1])
    ix.link_pivots(0, want_adjacency=False)
    ix.rng_build_exact()
    with pytest.raises(g.GrngError) as e:
        ix.rng_insert_batch(np.zeros((0, 8), np.float32))
    assert e.value.status == g.GRNG_EINVAL
