"""Lune-based beta-skeletons (rng_build_skeleton, 1 <= beta <= 2, L2) through the C ABI:
element by element against the FP64 oracle's brute force at a few thousand points (beta = 1
is the Gabriel graph, beta = 2 the RNG), on integer coordinates with ties and duplicates, and
at the mixture workload's full size (100,000 points) by sampled edges and non-edges checked
against every point in canonical FP64."""
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


def _skeleton(ix, beta):
    ix.rng_build_skeleton(beta)
    return ix.rng_edges()


@pytest.mark.parametrize("kind,n,precision", [("mix16", 2500, g.FP32), ("lin96", 1800, g.BF16)])
def test_skeletons_match_oracle(kind, n, precision):
    w = wl.make(kind, n=n)
    ix, out = g.build_all(w.X, w.layers, precision=precision)
    rng_edges = _es(out["edges"])
    prev = None
    for beta in (1.0, 1.25, 1.5, 1.75, 2.0):
        got = _es(_skeleton(ix, beta))
        assert got == _es(oracle.beta_skeleton(w.X, beta)), f"beta {beta}"
        assert rng_edges <= got                          # the RNG lies in every skeleton with beta <= 2
        if prev is not None:
            assert got <= prev                           # a larger beta keeps a subset
        prev = got
    assert prev == rng_edges                             # beta = 2 is the RNG
    assert ix.stats()["skeleton_beta"] == 2.0


def test_skeleton_ties_small_buffers():
    rng = np.random.default_rng(31)
    X = rng.integers(0, 5, size=(700, 3)).astype(np.float32)   # many equal keys and duplicates
    r2 = np.random.default_rng(32)
    fine = np.sort(r2.choice(700, 30, replace=False)).astype(np.int32)
    coarse = np.sort(r2.choice(fine, 5, replace=False)).astype(np.int32)
    ix, _ = g.build_all(X, [coarse, fine], flags=g.GRNG_FLAG_SMALL_BUFFERS, knn_k=4)
    for beta in (1.0, 1.5):
        assert _es(_skeleton(ix, beta)) == _es(oracle.beta_skeleton(X, beta)), f"beta {beta}"


def test_skeleton_errors_and_insertion():
    w = wl.make("uniform8", n=600)
    ix, _ = g.build_all(w.X[:500], [w.layers[-1][w.layers[-1] < 500]])
    for bad in (0.5, 2.5, float("nan")):
        with pytest.raises(g.GrngError) as e:
            ix.rng_build_skeleton(bad)
        assert e.value.status == g.GRNG_EINVAL
    ix.rng_build_skeleton(1.0)
    with pytest.raises(g.GrngError) as e:
        ix.rng_insert_batch(w.X[500:])                   # the stored graph is not the RNG
    assert e.value.status == g.GRNG_ESTATE
    ix.rng_build_exact()
    ix.rng_insert_batch(w.X[500:])
    assert _es(ix.rng_edges()) == _es(oracle.rng_brute(w.X))
    ixl, _ = g.build_all(w.X, w.layers, metric=g.L1)
    with pytest.raises(g.GrngError) as e:
        ixl.rng_build_skeleton(1.0)
    assert e.value.status == g.GRNG_EINVAL


def _keys_to(X64, i):
    """Canonical FP64 keys of every point to point i: the squared differences added in
    dimension order, each operation rounded (no fused multiply-add)."""
    acc = np.zeros(X64.shape[0])
    for d in range(X64.shape[1]):
        t = X64[:, d] - X64[i, d]
        acc = acc + t * t
    return acc


def _blocked(X64, i, j, beta):
    lam = beta / 2.0
    mu = 1.0 - lam
    a, b = _keys_to(X64, i), _keys_to(X64, j)
    v = a[j]
    t = lam * v
    inside = (mu * a + lam * b < t) & (lam * a + mu * b < t)
    inside[[i, j]] = False
    return bool(inside.any())


def test_gabriel_mixture_100k_sampled():
    w = wl.make("mix16")
    ix, out = g.build_all(torch.from_numpy(w.X).cuda(), w.layers)
    R = _es(out["edges"])
    E = _skeleton(ix, 1.0)
    assert np.all(E[:, 0] < E[:, 1])
    key = E[:, 0].astype(np.int64) * w.n + E[:, 1]
    assert np.all(np.diff(key) > 0), "edges not sorted or repeated"
    G = _es(E)
    assert R <= G and len(G) > len(R)
    X64 = w.X.astype(np.float64)
    rng = np.random.default_rng(33)
    for i, j in E[rng.choice(E.shape[0], size=200, replace=False)]:
        assert not _blocked(X64, int(i), int(j), 1.0), ("edge with a point inside", int(i), int(j))
    # non-edges among each point's 200 nearest: each must have a point strictly inside its
    # diametral ball (in 16 dimensions the first dozen neighbours are mostly Gabriel edges)
    checked = 0
    for i in rng.choice(w.n, size=40, replace=False):
        k = _keys_to(X64, int(i))
        k[int(i)] = np.inf
        for j in np.argsort(k)[:200:10]:
            a, b = min(int(i), int(j)), max(int(i), int(j))
            if (a, b) not in G:
                assert _blocked(X64, a, b, 1.0), ("non-edge without a blocker", a, b)
                checked += 1
    assert checked > 0
