"""The plain exact RNG at the mixture workload's full size (100,000 points in 16-D, 64
Gaussian clusters, pivot layers 256 and 4,096), L2 and L1, through the C ABI.

At this size the brute-force oracle (all triples) is out of reach, so the GPU result is
checked against what the definitions fix at any size:
  - each layer's assignment, radii and delta_max against the oracle (Eq. 2, Sec. 3);
  - each layer's GRNG against the oracle's definition (Sec. 2): all of the 256-pivot
    layer, 120 seeded rows of the 4,096-pivot one;
  - the exact RNG neighbourhoods of 400 seeded points against the oracle's rows (Eq. 1);
  - a minimum spanning tree of all points (Prim, FP64) lies in the RNG (Sec. 1), which
    also puts every point's nearest neighbour in it;
  - for L2, sampled RNG edges have empty diametral balls (RNG within the Gabriel graph);
  - every RNG edge joins members of equal or GRNG-linked finest domains (Theorem 1);
  - the edge list is sorted, i < j, without repeats.
"""
import numpy as np
import pytest

import oracle
from paper_2208_10022_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2208_10022_gb300 as g  # noqa: E402


def _rows_of(E, xs):
    both = np.concatenate([E, E[:, ::-1]])
    order = np.argsort(both[:, 0], kind="stable")
    src, dst = both[order, 0], both[order, 1]
    lo, hi = np.searchsorted(src, xs, "left"), np.searchsorted(src, xs, "right")
    return [np.sort(dst[lo[t]:hi[t]]) for t in range(len(xs))]


@pytest.mark.parametrize("metric", [wl.L2, wl.L1])
def test_mixture_100k_full_size(metric):
    w = wl.make("mix16", metric=metric)
    assert w.n == 100_000 and [len(l) for l in w.layers] == [256, 4096]
    ix, out = g.build_all(torch.from_numpy(w.X).cuda(), w.layers, metric=metric, want_adjacency=True)
    E = out["edges"]
    assert E.shape[0] > w.n - 1
    assert np.all(E[:, 0] < E[:, 1])
    key = E[:, 0].astype(np.int64) * w.n + E[:, 1]
    assert np.all(np.diff(key) > 0), "edges not sorted or repeated"
    # pivot layers: assignment, radii, delta_max and GRNG against the oracle
    lay = oracle.build_layers(w.X, w.layers, metric)
    for li in range(2):
        a, r, dm = out["layers"][li]
        assert np.array_equal(a, lay[li]["assign"]) and np.array_equal(r, lay[li]["radius"])
        assert np.array_equal(dm, lay[li]["delta_max"])
        off, adj = out["grng"][li]
        P = w.X[w.layers[li]]
        m = len(w.layers[li])
        if m <= 512:      # the whole GRNG by its definition
            Gw = oracle.grng_brute(P, lay[li]["radius"], metric)
            got = {(i, int(j)) for i in range(m) for j in adj[off[i]:off[i + 1]] if i < j}
            assert got == {tuple(map(int, e)) for e in Gw}, f"GRNG of layer {li}"
        else:             # seeded rows of it (the 4,096-pivot GRNG is nearly complete: O(m^3))
            for i in np.random.default_rng(3002 + li).choice(m, size=120, replace=False):
                want_row = oracle.grng_row(P, lay[li]["radius"], int(i), metric)
                assert np.array_equal(np.sort(adj[off[i]:off[i + 1]]), want_row), f"GRNG row {i} of layer {li}"
    # exact rows of seeded points
    xs = np.sort(np.random.default_rng(3001 + metric).choice(w.n, size=400, replace=False))
    want = oracle.rng_rows(w.X, xs, metric)
    got = _rows_of(E, xs)
    bad = [int(xs[t]) for t in range(len(xs)) if not np.array_equal(got[t], want[t])]
    assert not bad, f"{len(bad)} rows differ, e.g. point {bad[0]}"
    # a minimum spanning tree lies in the RNG
    T = oracle.emst(w.X, metric)
    tk = np.minimum(T[:, 0], T[:, 1]).astype(np.int64) * w.n + np.maximum(T[:, 0], T[:, 1])
    assert np.all(np.isin(tk, key)), f"{int((~np.isin(tk, key)).sum())} MST edges missing"
    # RNG within the Gabriel graph (L2): no point strictly inside the diametral ball
    if metric == wl.L2:
        X64 = w.X.astype(np.float64)
        for i, j in E[np.random.default_rng(3003).choice(E.shape[0], size=300, replace=False)]:
            kij = oracle.key(w.X[i], w.X[j])
            s = ((X64 - X64[i]) ** 2).sum(1) + ((X64 - X64[j]) ** 2).sum(1)
            s[[i, j]] = np.inf
            assert np.all(s >= kij * (1 - 1e-12)), ("GG", int(i), int(j))
    # Theorem 1: RNG edges only between equal or GRNG-linked finest domains
    a_f = out["layers"][1][0]
    off, adj = out["grng"][1]
    p, q = a_f[E[:, 0]], a_f[E[:, 1]]
    m = len(w.layers[1])
    linked = set()
    for i in range(m):
        for j in adj[off[i]:off[i + 1]]:
            linked.add(i * m + int(j))
    cross = p != q
    assert all((int(a) * m + int(b)) in linked for a, b in zip(p[cross], q[cross])), "Theorem 1"
