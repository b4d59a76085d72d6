"""The pivot-guided FP64 construction (the paper's stages, oracle/guided_oracle.c) against
the brute-force definition (Eq. 1 over all triples): two independent CPU routes to the
same RNG, on the configurations' generators, with one, two and three pivot layers, L2 and
L1, and on integer points with many exact ties and duplicates."""
import numpy as np
import pytest

import oracle
from paper_2208_10022_gb300 import workloads as wl


def _eq(a, b):
    return np.array_equal(np.asarray(a).reshape(-1, 2), np.asarray(b).reshape(-1, 2))


@pytest.mark.parametrize("kind,n,metric", [("uniform8", 1000, wl.L2), ("uniform8", 1000, wl.L1),
                                           ("mix16", 3000, wl.L2), ("mix16", 3000, wl.L1),
                                           ("lin96", 2000, wl.L2)])
def test_guided_equals_brute(kind, n, metric):
    w = wl.make(kind, n=n, metric=metric)
    E, st = oracle.rng_guided(w.X, w.layers, metric, with_stats=True)
    assert _eq(E, oracle.rng_brute(w.X, metric))
    # the guided route computes fewer distances than the N(N-1)/2 + triples of brute force
    assert st[0] > 0 and st[1] <= n * (n - 1) // 2


def test_guided_ties_duplicates_and_layer_counts():
    rng = np.random.default_rng(21)
    X = rng.integers(0, 5, size=(240, 3)).astype(np.float32)
    X[10] = X[3]
    X[50] = X[3]
    for metric in (wl.L2, wl.L1):
        want = oracle.rng_brute(X, metric)
        fine = np.sort(rng.choice(240, 48, replace=False)).astype(np.int32)
        mid = np.sort(rng.choice(fine, 12, replace=False)).astype(np.int32)
        top = np.sort(rng.choice(mid, 3, replace=False)).astype(np.int32)
        for layers in ([fine], [mid, fine], [top, mid, fine]):
            assert _eq(oracle.rng_guided(X, layers, metric), want), (metric, len(layers))


def test_candidate_rules_sound_and_restated():
    """Stage I candidates under the nearest-pivot rule (per-pivot radii) and under the paper's
    uniform radius with every pivot within r a parent: both keep every RNG edge (Theorem 1),
    and each candidate set equals its restatement through the definitions' oracle functions
    (assignment, GRNG by its definition)."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(41)
    for t in range(10):
        n = int(rng.integers(40, 110))
        if t < 4:  # dense pivots on a line or a plane: sparse GRNGs, several parents per point
            d = 1 + t // 2
            piv = np.sort(rng.choice(n, n // 4, replace=False)).astype(np.int32)
        else:
            d = int(rng.integers(2, 5))
            piv = np.sort(rng.choice(n, int(rng.integers(4, 12)), replace=False)).astype(np.int32)
        X = rng.standard_normal((n, d)).astype(np.float32)
        for metric in (oracle.L2, oracle.L1):
            dist = np.array([[oracle.dist(X[i], X[p], metric) for p in piv] for i in range(n)])
            promote = t % 2 == 1
            r = float(dist.min(1).max()) * (0.6 if promote else 1.0)
            res = oracle.candidate_rules(X, piv, r, metric, want_sets=True, promote=promote)
            E = {tuple(e) for e in oracle.rng_brute(X, metric).tolist()}
            assert E <= res["set_a"] and E <= res["set_b"], (t, metric)
            a, _, rad, _ = oracle.assign(X, np.arange(n), piv, metric=metric)
            G = {tuple(e) for e in oracle.grng_brute(X[piv], rad, metric).tolist()}
            want_a = {(i, j) for i in range(n) for j in range(i + 1, n)
                      if a[i] == a[j] or (min(a[i], a[j]), max(a[i], a[j])) in G}
            assert res["set_a"] == want_a, (t, metric)
            if not promote:
                assert res["no_parent"] == 0 and res["pivots_b"] == len(piv)
                GB = {tuple(e) for e in oracle.grng_brute(X[piv], np.full(len(piv), r), metric).tolist()}
                par = [[p for p in range(len(piv)) if dist[i, p] <= r] for i in range(n)]
                want_b = {(i, j) for i in range(n) for j in range(i + 1, n)
                          if all(p == q or (min(p, q), max(p, q)) in GB for p in par[i] for q in par[j])}
                assert res["set_b"] == want_b, (t, metric)
            else:
                assert res["no_parent"] == 0 and res["pivots_b"] >= len(piv)


def test_search_by_stages_equals_definition():
    """RNG search by the paper's Stages I-VI (Theorem 1, the virtual-pivot prunes of Stages II
    and III, pivots and members as interceptors) returns exactly the definition's neighbours,
    on random points (L2, L1) and on small integers with ties and duplicates."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(43)
    for t in range(8):
        n = int(rng.integers(150, 500))
        d = int(rng.integers(1, 5))
        if t % 4 == 3:
            X = rng.integers(0, 5, size=(n, d)).astype(np.float32)
            Q = np.concatenate([rng.integers(0, 5, size=(20, d)), X[:3]]).astype(np.float32)
        else:
            X = rng.standard_normal((n, d)).astype(np.float32)
            Q = np.concatenate([rng.standard_normal((20, d)) * 1.3, X[:3], X[:1] * 9.0]).astype(np.float32)
        piv = np.sort(rng.choice(n, int(rng.integers(5, 40)), replace=False)).astype(np.int32)
        for metric in (oracle.L2, oracle.L1):
            got, st = oracle.rng_search_guided(X, piv, Q, metric)
            want = oracle.rng_search(X, Q, metric)
            bad = [j for j in range(len(Q)) if not np.array_equal(got[j], want[j])]
            assert not bad, (t, metric, bad[:3])
            assert st["after_stage3"] <= st["after_stage2"] <= st["after_stage1"] <= n * len(Q)


def test_search_by_stages_on_the_workload_generators():
    """The two search routes agree on the mixture and lin96 generators (three pivot counts)."""
    import numpy as np

    import oracle
    from paper_2208_10022_gb300 import workloads as wl
    for kind, n in (("mix16", 1500), ("lin96", 1200)):
        allp = wl.gen_points(kind, n + 12, 77)
        X, Q = allp[:n], allp[n:]
        for m in (8, 40, 160):
            piv = wl.nested_pivots(n, [m], 5 + m)[0]
            got, _ = oracle.rng_search_guided(X, piv, Q)
            want = oracle.rng_search(X, Q)
            assert all(np.array_equal(a, b) for a, b in zip(got, want)), (kind, m)
