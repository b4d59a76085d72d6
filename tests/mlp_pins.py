"""Pins of the FP64 interceptor-ranking network in oracle/mlp_oracle.c.

Each check takes the oracle module and raises AssertionError on a mismatch.  None of
them re-types the oracle's formulas: the forward pass is pinned by networks whose
output has a closed form, the gradient by central finite differences of the loss
(which only calls the forward-and-loss path) and by closed forms of the output-layer
gradient.
"""
import numpy as np

IN, H = 32, 128
OFF_W1 = 0
OFF_B1 = OFF_W1 + H * IN
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
NP = OFF_B3 + 1


def _copy_net(c):
    """First layer copies the 32 inputs, second copies them again, output sums them:
    s = c + sum_k relu(f_k)."""
    P = np.zeros(NP)
    for k in range(IN):
        P[OFF_W1 + k * IN + k] = 1.0
        P[OFF_W2 + k * H + k] = 1.0
        P[OFF_W3 + k] = 1.0
    P[OFF_B3] = c
    return P


def pin_parameter_count(orc):
    assert orc.mlp_nparams() == NP == 20865


def pin_forward_copy_network(orc):
    rng = np.random.default_rng(11)
    X = rng.normal(size=(50, IN))
    s = orc.mlp_forward(_copy_net(0.25), X)
    want = 0.25 + np.maximum(X, 0.0).sum(axis=1)
    assert np.allclose(s, want, rtol=0, atol=1e-12), np.abs(s - want).max()


def pin_forward_weighted_unit(orc):
    """One hidden path: h1_0 = relu(a.f + b), h2_0 = relu(2 h1_0 - 1), s = 3 h2_0 - 0.5."""
    rng = np.random.default_rng(12)
    a = rng.normal(size=IN)
    P = np.zeros(NP)
    P[OFF_W1:OFF_W1 + IN] = a
    P[OFF_B1] = 0.3
    P[OFF_W2] = 2.0
    P[OFF_B2] = -1.0
    P[OFF_W3] = 3.0
    P[OFF_B3] = -0.5
    X = rng.normal(size=(64, IN))
    h1 = np.maximum(X @ a + 0.3, 0.0)
    want = 3.0 * np.maximum(2.0 * h1 - 1.0, 0.0) - 0.5
    s = orc.mlp_forward(P, X)
    assert np.allclose(s, want, rtol=1e-13, atol=1e-13)


def pin_loss_constant_network(orc):
    """All weights zero: s = b3 for every sample, L = mean w (softplus(b3) - y b3) and
    dL/db3 = mean w (sigmoid(b3) - y); every other gradient is zero."""
    P = np.zeros(NP)
    P[OFF_B3] = 0.7
    rng = np.random.default_rng(13)
    X = rng.normal(size=(40, IN))
    y = (rng.random(40) < 0.3).astype(float)
    w = rng.random(40) + 0.5
    loss, g = orc.mlp_loss_grad(P, X, y, w)
    sp = np.log1p(np.exp(0.7))
    assert abs(loss - np.mean(w * (sp - y * 0.7))) < 1e-13
    assert abs(g[OFF_B3] - np.mean(w * (1 / (1 + np.exp(-0.7)) - y))) < 1e-13
    assert np.all(g[:OFF_B3] == 0.0)


def pin_output_layer_gradient(orc):
    """With W2 = 0 and b2 > 0, h2 = b2 for every sample: dL/dw3 = mean(ds) b2 with
    ds = w (sigmoid(s) - y), and the layers below get no gradient through w3 . h2's
    constant input."""
    rng = np.random.default_rng(14)
    P = np.zeros(NP)
    b2 = rng.random(H) + 0.1
    P[OFF_B2:OFF_B2 + H] = b2
    P[OFF_W3:OFF_W3 + H] = rng.normal(size=H) * 0.1
    P[OFF_B3] = -0.2
    X = rng.normal(size=(30, IN))
    y = (rng.random(30) < 0.5).astype(float)
    loss, g = orc.mlp_loss_grad(P, X, y)
    s = b2 @ P[OFF_W3:OFF_W3 + H] - 0.2
    ds = 1 / (1 + np.exp(-s)) - y
    assert np.allclose(g[OFF_W3:OFF_W3 + H], ds.mean() * b2, rtol=1e-12, atol=1e-14)
    assert np.allclose(g[OFF_B2:OFF_B2 + H], ds.mean() * P[OFF_W3:OFF_W3 + H], rtol=1e-12, atol=1e-14)
    assert np.all(g[OFF_W2:OFF_B2] == 0.0)


def pin_finite_differences(orc):
    """Central differences of the loss against the analytic gradient, for parameters of
    every block, at a random point away from the rectifier kinks."""
    rng = np.random.default_rng(15)
    P = rng.normal(size=NP) * 0.2
    X = rng.normal(size=(24, IN))
    y = (rng.random(24) < 0.4).astype(float)
    w = rng.random(24) + 0.5
    _, g = orc.mlp_loss_grad(P, X, y, w)
    idx = np.concatenate([rng.integers(lo, hi, 12) for lo, hi in
                          ((OFF_W1, OFF_B1), (OFF_B1, OFF_W2), (OFF_W2, OFF_B2), (OFF_B2, OFF_W3),
                           (OFF_W3, OFF_B3))] + [np.array([OFF_B3])])
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (orc.mlp_loss_grad(Pp, X, y, w)[0] - orc.mlp_loss_grad(Pm, X, y, w)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (int(i), fd, g[i])


ALL = [pin_parameter_count, pin_forward_copy_network, pin_forward_weighted_unit, pin_loss_constant_network,
       pin_output_layer_gradient, pin_finite_differences]
