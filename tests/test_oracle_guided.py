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
