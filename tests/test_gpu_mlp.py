"""The learned shortlist on the GPU, through the C ABI:

  - the FP32 gradient of the ranking network against the FP64 oracle's;
  - BF16-weight scoring against the oracle's forward pass with the same rounded weights;
  - training lowers the loss;
  - a build with the shortlist switched on gives the oracle's edge set (it only changes
    which interceptors are tried first);
  - the gain: a network trained on samples recorded from a 200,000-point build cuts the
    exhaustive-tier interceptor evaluations of another 200,000-point build, and blocks
    more pairs than the same network untrained.
"""
import numpy as np
import pytest

import oracle
from paper_2208_10022_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # collected on CPU machines, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2208_10022_gb300 as g  # noqa: E402


def _bf16(a):
    """Round float32 values to BF16 (nearest, ties to even), back as float32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 32)).astype(np.float32)
    y = (rng.random(n) < 0.3).astype(np.float32)
    w = (rng.random(n) + 0.5).astype(np.float32)
    return X, y, w


def test_gradient_matches_oracle():
    P = (g.mlp_init(3) * 0.8).astype(np.float32)
    P[4096:4224] = 0.05  # b1
    X, y, w = _samples(512, 4)
    loss, grad = g.mlp_loss_grad(P, X, y, w)
    l64, g64 = oracle.mlp_loss_grad(P.astype(np.float64), X, y, w)
    assert abs(loss - l64) <= 1e-5 * max(1.0, abs(l64))
    scale = np.abs(g64).max()
    err = np.abs(grad.astype(np.float64) - g64)
    assert err.max() <= 2e-4 * scale, (err.max(), scale)
    # every block of parameters is exercised
    assert np.count_nonzero(g64) > 0.5 * g64.size


def test_bf16_scores_match_oracle():
    P = g.mlp_init(5)
    P[-1] = 0.3
    X, _, _ = _samples(1000, 6)
    got = g.mlp_score(P, X).astype(np.float64)
    Pr = P.copy()
    n_w1, n_w2 = 128 * 32, 128 * 128
    Pr[:n_w1] = _bf16(P[:n_w1])                              # W1
    Pr[n_w1 + 128:n_w1 + 128 + n_w2] = _bf16(P[n_w1 + 128:n_w1 + 128 + n_w2])  # W2
    want = oracle.mlp_forward(Pr.astype(np.float64), X)
    err = np.abs(got - want)
    assert err.max() <= 1e-4 * (1.0 + np.abs(want).max()), err.max()


def test_training_lowers_the_loss():
    rng = np.random.default_rng(7)
    X = rng.normal(size=(20000, 32)).astype(np.float32)
    y = ((X[:, 0] - 0.5 * X[:, 3] + 0.25 * X[:, 7]) > 0.2).astype(np.float32)
    P0 = g.mlp_init(8)
    l0, _ = g.mlp_loss_grad(P0, X, y)
    P1, last = g.mlp_train(P0, X, y, epochs=8, batch=1024, lr=2e-3)
    l1, _ = g.mlp_loss_grad(P1, X, y)
    assert l1 < 0.25 * l0 and l1 < 0.15, (l0, l1, last)
    acc = np.mean((g.mlp_score(P1, X) > 0) == (y > 0.5))
    assert acc > 0.95


@pytest.mark.parametrize("kind,metric,n", [("lin96", wl.L2, 2500), ("mix16", wl.L1, 1500)])
def test_shortlist_build_matches_oracle(kind, metric, n):
    # one-entry neighbour lists leave many pairs to the exhaustive tier
    w = wl.make(kind, n=n, metric=metric)
    P = g.mlp_init(9)
    ix, out = g.build_all(w.X, w.layers, metric=metric, knn_k=1, mlp_params=P, k_shortlist=8)
    st = ix.stats()["rng"]
    assert st["learned_pairs"] == st["tier3_pairs"]
    if metric == wl.L2:
        assert st["tier3_pairs"] > 0 and st["learned_candidates"] > 0 and st["learned_tests"] > 0
    got = {tuple(e) for e in out["edges"].tolist()}
    want = {tuple(e) for e in oracle.rng_brute(w.X, metric).tolist()}
    assert got == want


def _tier3_evals(st):
    return st["tier3_nodes_tested"] + st.get("learned_tests", 0)


def test_trained_shortlist_gain():
    # training samples from one 200,000-point build of the lin96 generator
    wt = wl.make("lin96", n=200000)
    ix, _ = g.build_all(wt.X, wt.layers, flags=g.GRNG_FLAG_RECORD_MLP)
    F, y = ix.mlp_dataset()
    st_t = ix.stats()["rng"]
    ix.close()
    print(f"\ntraining build: {F.shape[0]} samples, {int(y.sum())} positive; tier-3 pairs {st_t['tier3_pairs']}, "
          f"blocked {st_t['tier3_blocked']}, with a blocker in the pool {st_t['learned_pool_hits']}")
    assert F.shape[0] > 10000 and 0 < y.sum() < y.size
    pos = y.mean()
    wts = np.where(y > 0.5, 0.5 / pos, 0.5 / (1.0 - pos)).astype(np.float32)
    perm = np.random.default_rng(10).permutation(F.shape[0])
    P0 = g.mlp_init(11)
    P1, _ = g.mlp_train(P0, F[perm], y[perm], wts[perm], epochs=6, batch=4096, lr=1e-3)
    # evaluation on another draw of the same generator
    we = wl.make("lin96", n=200000, data_seed=4242, pivot_seed=4343)
    ix0, out0 = g.build_all(we.X, we.layers)
    s0 = ix0.stats()["rng"]
    ixr, outr = g.build_all(we.X, we.layers, mlp_params=P0, k_shortlist=8)
    sr = ixr.stats()["rng"]
    ix1, out1 = g.build_all(we.X, we.layers, mlp_params=P1, k_shortlist=8)
    s1 = ix1.stats()["rng"]
    e0 = {tuple(e) for e in out0["edges"].tolist()}
    assert {tuple(e) for e in out1["edges"].tolist()} == e0
    assert {tuple(e) for e in outr["edges"].tolist()} == e0
    assert s1["tier3_pairs"] == s0["tier3_pairs"] > 0
    print(f"\ntier-3 pairs {s0['tier3_pairs']}, blocked {s0['tier3_blocked']}; shortlist blocks: "
          f"trained {s1['learned_blocked']}, untrained {sr['learned_blocked']}; interceptor evaluations "
          f"without {_tier3_evals(s0)}, trained {_tier3_evals(s1)}, untrained {_tier3_evals(sr)}")
    assert s1["learned_blocked"] > sr["learned_blocked"]
    assert _tier3_evals(s1) < _tier3_evals(s0)
