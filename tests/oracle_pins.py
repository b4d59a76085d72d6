"""Pins of the FP64 oracle to facts outside itself.

Each check takes the oracle binding as an argument so the same checks can be run
against deliberately broken builds of the oracle (see test_oracle_mutants.py).
Every check raises AssertionError on failure.

What pins what:
  exact_rng / exact_grng   -- Eq. 1 and the GRNG definition in exact rational
                              arithmetic on tiny integer/dyadic inputs (exhaustive)
  worked_examples          -- hand-derived edge sets (tests/golden)
  invariants               -- 1NN within MST within RNG within GG (Sec. 1), GRNG
                              with zero radii = RNG, GRNG contains RNG(P) and is
                              connected (Sec. 2), Theorem 1 and Theorem 2 as
                              properties of the oracle's outputs
  cross_checks             -- rng_row vs rng_brute and grng_row vs grng_brute (two
                              different loops), assignment vs a Python restatement
  layer_examples           -- a hand-derived two-layer hierarchy whose coarse radius
                              and delta_max differ (tests/golden)
  witnesses                -- the witness check against the exact lune test, and
                              every non-edge of Eq. 1 has a witness
  spanning_trees           -- Prim's tree has the weight of an exact Kruskal over all
                              pairs and lies in the RNG
  skeletons                -- beta-skeletons (1 <= beta <= 2) against the exact rational
                              predicate, beta = 1 against the Gabriel graph from the
                              midpoint, beta = 2 against the RNG, and nesting in beta
  pivot_insertion          -- the GRNG after a new pivot joins (its Stage VII) against the
                              definition's GRNG of all pivots
  search                   -- RNG search (Algorithm 1 without Stage VII) against the exact
                              rational restatement, against the brute-force RNG of the
                              index plus that one query, and batch = one query at a time
"""
import json
import os

import numpy as np

from . import exact

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "worked_examples.json")
LAYERS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "layers_delta_max.json")


def _as_set(E):
    return {tuple(map(int, e)) for e in np.asarray(E).reshape(-1, 2)}


def _rand_int_points(rng, n, d, hi):
    return rng.integers(0, hi + 1, size=(n, d)).astype(np.float32)


def exact_rng(orc, trials=60, seed=11):
    rng = np.random.default_rng(seed)
    for t in range(trials):
        n = int(rng.integers(3, 11))
        d = int(rng.integers(1, 4))
        X = _rand_int_points(rng, n, d, 4)          # small integers: many exact ties
        for metric in (exact.L2, exact.L1):
            want = set(exact.rng(X.tolist(), metric))
            got = _as_set(orc.rng_brute(X, metric))
            assert got == want, (t, metric, X.tolist(), sorted(want ^ got))


def exact_grng(orc, trials=60, seed=12):
    rng = np.random.default_rng(seed)
    for t in range(trials):
        m = int(rng.integers(3, 10))
        d = int(rng.integers(1, 4))
        P = _rand_int_points(rng, m, d, 6)
        for metric in (exact.L2, exact.L1):
            r = rng.integers(0, 5, size=m) / 8.0          # dyadic radii, exact in FP64
            if t % 5 == 0:
                r[:] = 0.0
            want = set(exact.grng(P.tolist(), r.tolist(), metric))
            got = _as_set(orc.grng_brute(P, r, metric))
            assert got == want, (t, metric, P.tolist(), r.tolist(), sorted(want ^ got))


def worked_examples(orc):
    g = json.load(open(GOLDEN))
    for ex in g["rng"]:
        X = np.asarray(ex["points"], np.float32)
        assert _as_set(orc.rng_brute(X, ex["metric"])) == _as_set(ex["edges"]), ex["name"]
    for ex in g["grng"]:
        P = np.asarray(ex["points"], np.float32)
        r = np.asarray(ex["radii"], np.float64)
        assert _as_set(orc.grng_brute(P, r, ex["metric"])) == _as_set(ex["edges"]), ex["name"]


def _key_matrix(orc, X, metric):
    n = X.shape[0]
    K = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            K[i, j] = K[j, i] = orc.key(X[i], X[j], metric)
    return K


def _mst_edges(K):
    """Kruskal on the FP64 key matrix (any MST lies in the RNG: the lune is open)."""
    n = K.shape[0]
    iu = np.triu_indices(n, 1)
    order = np.argsort(K[iu], kind="stable")
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    out = set()
    for t in order:
        i, j = int(iu[0][t]), int(iu[1][t])
        a, b = find(i), find(j)
        if a != b:
            parent[a] = b
            out.add((i, j))
    return out


def _connected(n, E):
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for i, j in E:
        parent[find(i)] = find(j)
    return len({find(i) for i in range(n)}) == 1


def invariants(orc, seed=13):
    rng = np.random.default_rng(seed)
    for t in range(6):
        n = int(rng.integers(40, 160))
        d = int(rng.integers(2, 7))
        X = rng.standard_normal((n, d)).astype(np.float32)
        for metric in (exact.L2, exact.L1):
            E = _as_set(orc.rng_brute(X, metric))
            K = _key_matrix(orc, X, metric)
            assert all(i < j for i, j in E)
            # 1NN within RNG (Sec. 1 chain)
            Kd = K + np.diag(np.full(n, np.inf))
            for i in range(n):
                j = int(np.argmin(Kd[i]))
                assert (min(i, j), max(i, j)) in E, ("1NN", i, j)
            # MST within RNG, hence connected (Sec. 1)
            assert _mst_edges(K) <= E
            assert _connected(n, E)
            if metric == exact.L2:
                # RNG within the Gabriel graph (Sec. 1)
                for i, j in E:
                    s = K[i] + K[j]
                    s[i] = s[j] = np.inf
                    assert np.all(s >= K[i, j]), ("GG", i, j)
            # GRNG with zero radii is the RNG; radii >= 0 only add links (Sec. 2)
            assert _as_set(orc.grng_brute(X, np.zeros(n), metric)) == E
            r = rng.uniform(0, 0.3, size=n)
            G = _as_set(orc.grng_brute(X, r, metric))
            assert E <= G and _connected(n, G)
            # closed form: once d_ij <= 3 (r_i + r_j) for every pair, no pivot can block
            dmax = np.sqrt(K.max()) if metric == exact.L2 else K.max()
            big = np.full(n, dmax / 6.0 * 1.01)
            assert len(_as_set(orc.grng_brute(X, big, metric))) == n * (n - 1) // 2


def theorems(orc, seed=14):
    """Theorem 1 and Theorem 2 as properties of the oracle's own outputs."""
    rng = np.random.default_rng(seed)
    for t in range(4):
        n = int(rng.integers(200, 400))
        X = rng.standard_normal((n, 3)).astype(np.float32)
        for metric in (exact.L2, exact.L1):
            fine = np.sort(rng.choice(n, size=n // 8, replace=False)).astype(np.int32)
            coarse = np.sort(rng.choice(fine, size=max(2, len(fine) // 6), replace=False)).astype(np.int32)
            lay = orc.build_layers(X, [coarse, fine], metric)
            a_f = lay[1]["assign"]
            G_f = _as_set(orc.grng_brute(X[fine], lay[1]["radius"], metric))
            E = _as_set(orc.rng_brute(X, metric))
            # Theorem 1: RNG links only between members of equal or GRNG-linked domains
            for x, y in E:
                p, q = sorted((int(a_f[x]), int(a_f[y])))
                assert p == q or (p, q) in G_f, ("Thm1", x, y)
            # Theorem 2: fine GRNG links only between children of equal or linked coarse pivots
            a_c = lay[0]["assign"]
            G_c = _as_set(orc.grng_brute(X[coarse], lay[0]["radius"], metric))
            for i, j in G_f:
                p, q = sorted((int(a_c[i]), int(a_c[j])))
                assert p == q or (p, q) in G_c, ("Thm2", i, j)
            # relative pivot domains nest (Sec. 3): d(c, pb) <= R_c - rb
            R = lay[0]["radius"]
            for t_, pb in enumerate(fine):
                c = coarse[a_c[t_]]
                dd = orc.dist(X[c], X[pb], metric)
                assert dd + lay[1]["radius"][t_] <= R[a_c[t_]]


def cross_checks(orc, seed=15):
    rng = np.random.default_rng(seed)
    for t in range(3):
        n = int(rng.integers(100, 300))
        X = rng.standard_normal((n, 4)).astype(np.float32)
        for metric in (exact.L2, exact.L1):
            E = _as_set(orc.rng_brute(X, metric))
            for x in rng.choice(n, size=12, replace=False):
                want = sorted({j for i, j in E if i == x} | {i for i, j in E if j == x})
                assert list(orc.rng_row(X, x, metric)) == want, ("row", x)
            r = rng.uniform(0, 0.2, size=n)
            r[rng.random(n) < 0.3] = 0.0
            G = _as_set(orc.grng_brute(X, r, metric))
            for i in rng.choice(n, size=12, replace=False):
                want = sorted({j for a, j in G if a == i} | {a for a, j in G if j == i})
                assert list(orc.grng_row(X, r, i, metric)) == want, ("grow", i)
    # assignment against a Python restatement in the same canonical order
    X = rng.standard_normal((120, 5)).astype(np.float32)
    X[7] = X[3]                                    # a duplicate of a pivot
    piv = np.array([3, 10, 20, 30, 7], np.int32)   # 7 duplicates pivot 3, at a higher position
    for metric in (exact.L2, exact.L1):
        a, d, r, dm = orc.assign(X, np.arange(120, dtype=np.int32), piv, None, metric)
        for x in range(120):
            keys = []
            for p in piv:
                acc = 0.0
                for k in range(5):
                    t_ = float(X[x, k]) - float(X[p, k])
                    acc = acc + (t_ * t_ if metric == exact.L2 else abs(t_))
                keys.append(acc)
            if x in piv:
                want = int(np.where(piv == x)[0][0])
            else:
                want = int(np.argmin(keys))         # first minimum = lowest position
            assert a[x] == want, (x, a[x], want)
        for p in range(len(piv)):
            mem = np.where(a == p)[0]
            assert r[p] == (d[mem].max() if len(mem) else 0.0)
            assert dm[p] == r[p]
        assert a[7] == 4 and a[3] == 0


def degree_arithmetic():
    """Table 4's average degrees are 2E/N; the bench reports degree the same way."""
    g = json.load(open(GOLDEN))
    for ex in g["degree"]:
        assert round(2.0 * ex["edges"] / ex["n"], 4) == ex["avg_degree"], ex["name"]


def layer_examples(orc):
    """Assignment, radius and delta_max of both layers equal the hand-derived values."""
    g = json.load(open(LAYERS))
    X = np.asarray(g["points"], np.float32)
    for case in g["cases"]:
        lay = orc.build_layers(X, [np.asarray(l, np.int32) for l in g["layers"]], case["metric"])
        for li in range(len(g["layers"])):
            assert list(lay[li]["assign"]) == case["assign"][li], ("assign", case["metric"], li)
            assert list(lay[li]["radius"]) == case["radius"][li], ("radius", case["metric"], li)
            assert list(lay[li]["delta_max"]) == case["delta_max"][li], ("delta_max", case["metric"], li)


def witnesses(orc, trials=25, seed=16):
    """verify_witness(x, y, z) is the exact rational lune test; a pair is a non-edge of
    Eq. 1 exactly when some z is a witness."""
    rng = np.random.default_rng(seed)
    for t in range(trials):
        n = int(rng.integers(3, 9))
        d = int(rng.integers(1, 4))
        X = _rand_int_points(rng, n, d, 4)
        for metric in (exact.L2, exact.L1):
            E = set(exact.rng(X.tolist(), metric))
            for i in range(n):
                for j in range(i + 1, n):
                    any_w = False
                    for k in range(n):
                        kij = exact.key(X[i].tolist(), X[j].tolist(), metric)
                        inside = k not in (i, j) and max(exact.key(X[k].tolist(), X[i].tolist(), metric),
                                                         exact.key(X[k].tolist(), X[j].tolist(), metric)) < kij
                        w = orc.verify_witness(X, i, j, k, metric)
                        assert w == inside, (t, metric, i, j, k)
                        any_w |= w
                    assert any_w == ((i, j) not in E), (t, metric, i, j)


def spanning_trees(orc, seed=17):
    """Prim's tree (orc.emst) is a spanning tree with the weight of Kruskal's over the
    exact key matrix, and every tree edge is an RNG edge (Sec. 1: MST within RNG)."""
    rng = np.random.default_rng(seed)
    for t in range(4):
        n = int(rng.integers(30, 120))
        X = rng.standard_normal((n, 3)).astype(np.float32)
        for metric in (exact.L2, exact.L1):
            T = orc.emst(X, metric)
            assert T.shape == (n - 1, 2) and _connected(n, [tuple(map(int, e)) for e in T])
            K = _key_matrix(orc, X, metric)
            w_prim = sum(K[int(a), int(b)] for a, b in T)
            w_kruskal = sum(K[i, j] for i, j in _mst_edges(K))
            assert abs(w_prim - w_kruskal) <= 1e-9 * max(1.0, w_kruskal), (t, metric)
            E = _as_set(orc.rng_brute(X, metric))
            assert {(min(int(a), int(b)), max(int(a), int(b))) for a, b in T} <= E


def search(orc, trials=30, seed=18):
    rng = np.random.default_rng(seed)
    for t in range(trials):  # exact arithmetic on small integers: ties and duplicates
        n = int(rng.integers(2, 10))
        d = int(rng.integers(1, 4))
        X = _rand_int_points(rng, n, d, 4)
        Q = np.concatenate([_rand_int_points(rng, 3, d, 4), X[:1]])  # the last one duplicates x0
        for metric in (exact.L2, exact.L1):
            want = exact.rng_search(X.tolist(), Q.tolist(), metric)
            got = [list(map(int, r)) for r in orc.rng_search(X, Q, metric)]
            assert got == want, (t, metric, X.tolist(), Q.tolist(), want, got)
    # a query alone: its neighbours are its edges in the RNG of the index plus it (Eq. 1)
    for t in range(6):
        X = rng.normal(size=(120, 5)).astype(np.float32)
        Q = rng.normal(size=(8, 5)).astype(np.float32) * 1.5
        Q[0] = X[7]                                               # a duplicate of an index point
        for metric in (exact.L2, exact.L1):
            got = orc.rng_search(X, Q, metric)
            for j in range(len(Q)):
                E = orc.rng_brute(np.concatenate([X, Q[j:j + 1]]), metric)
                want = sorted(int(a) for a, b in E if b == len(X))
                assert list(map(int, got[j])) == want, (t, metric, j)
                assert list(map(int, orc.rng_search(X, Q[j:j + 1], metric)[0])) == want  # alone = in a batch
            assert 7 in set(map(int, got[0]))                        # a duplicate is always linked


def skeletons(orc, trials=30, seed=19):
    from fractions import Fraction
    rng = np.random.default_rng(seed)
    for t in range(trials):  # small integers: exact ties
        n = int(rng.integers(3, 10))
        d = int(rng.integers(1, 4))
        X = _rand_int_points(rng, n, d, 4)
        for beta in (Fraction(1), Fraction(5, 4), Fraction(3, 2), Fraction(2)):
            want = set(exact.beta_skeleton(X.tolist(), beta / 2))
            got = _as_set(orc.beta_skeleton(X, float(beta)))
            assert got == want, (t, float(beta), X.tolist(), sorted(want ^ got))
        assert _as_set(orc.beta_skeleton(X, 1.0)) == set(exact.gabriel(X.tolist())), (t, X.tolist())
    for t in range(4):  # beta = 2 is the RNG; a larger beta keeps a subset of the edges
        X = rng.standard_normal((90, 4)).astype(np.float32)
        E = [_as_set(orc.beta_skeleton(X, b)) for b in (1.0, 1.25, 1.5, 1.75, 2.0)]
        assert E[-1] == _as_set(orc.rng_brute(X, exact.L2))
        assert all(E[k + 1] <= E[k] for k in range(len(E) - 1))
        assert len(E[0]) > len(E[-1])


def pivot_insertion(orc, trials=12, seed=20):
    """Stage VII of the GRNG: the links after a new pivot joins equal the definition's GRNG of
    all pivots, for dyadic and zero radii, both metrics."""
    rng = np.random.default_rng(seed)
    pruned = 0
    for t in range(trials):
        m = int(rng.integers(6, 40))
        d = int(rng.integers(1, 4))
        P = rng.standard_normal((m + 1, d)).astype(np.float32)
        r = rng.integers(0, 3, size=m + 1) / 16.0 if t % 3 else np.zeros(m + 1)
        for metric in (exact.L2, exact.L1):
            old = orc.grng_brute(P[:m], r[:m], metric)
            got, (tested, removed, added) = orc.grng_insert_pivot(P, r, old, metric)
            want = _as_set(orc.grng_brute(P, r, metric))
            assert _as_set(got) == want, (t, metric)
            assert removed == len(_as_set(old) - want) and added == sum(1 for e in want if e[1] == m)
            pruned += len(old) - tested
    assert pruned > 0  # the longest-link bound skips some links


ALL = [exact_rng, exact_grng, worked_examples, invariants, theorems, cross_checks, layer_examples, witnesses,
       spanning_trees, search, skeletons, pivot_insertion]
