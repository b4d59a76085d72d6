"""Exact rational restatement of Eq. 1 (RNG) and of the GRNG definition (Sec. 2).

Python `fractions` arithmetic, no rounding anywhere: used to pin the FP64 oracle on
tiny inputs whose coordinates and radii are exactly representable.  L2 comparisons
that involve a square root are decided by exact algebra on the squared values.
"""
from fractions import Fraction as F
from itertools import combinations

L2, L1 = 0, 1


def key(a, b, metric):
    if metric == L2:
        return sum((F(x) - F(y)) ** 2 for x, y in zip(a, b))
    return sum(abs(F(x) - F(y)) for x, y in zip(a, b))


def rng(X, metric):
    """Edges (i<j) of the RNG by Eq. 1 (x3 ranges over S minus {x1, x2})."""
    n = len(X)
    K = [[key(X[i], X[j], metric) for j in range(n)] for i in range(n)]
    out = []
    for i, j in combinations(range(n), 2):
        if not any(max(K[k][i], K[k][j]) < K[i][j] for k in range(n) if k not in (i, j)):
            out.append((i, j))
    return out


def rng_search(X, Q, metric):
    """For each query q of Q, the index points x of X (ascending) with no index point z
    other than x strictly inside the open lune of (q, x): Eq. 1 over X plus q alone."""
    out = []
    for q in Q:
        kq = [key(q, x, metric) for x in X]
        row = []
        for i, x in enumerate(X):
            if not any(max(kq[k], key(X[k], x, metric)) < kq[i] for k in range(len(X)) if k != i):
                row.append(i)
        out.append(row)
    return out


def beta_skeleton(X, lam):
    """Edges (i<j) of the lune-based beta-skeleton (L2), lam = beta / 2 a Fraction in [1/2, 1]:
    z blocks (x, y) iff (1-lam) a + lam b < lam v and lam a + (1-lam) b < lam v (squared
    distances a = |z-x|^2, b = |z-y|^2, v = |x-y|^2)."""
    n = len(X)
    lam = F(lam)
    K = [[key(X[i], X[j], L2) for j in range(n)] for i in range(n)]
    out = []
    for i, j in combinations(range(n), 2):
        v = K[i][j]
        if not any((1 - lam) * K[k][i] + lam * K[k][j] < lam * v and lam * K[k][i] + (1 - lam) * K[k][j] < lam * v
                   for k in range(n) if k not in (i, j)):
            out.append((i, j))
    return out


def gabriel(X):
    """Edges (i<j) of the Gabriel graph from coordinates: no z strictly inside the ball with
    diameter xy, i.e. |2z - x - y|^2 < |x - y|^2."""
    n = len(X)
    out = []
    for i, j in combinations(range(n), 2):
        xi, xj = [F(t) for t in X[i]], [F(t) for t in X[j]]
        dd = sum((a - b) ** 2 for a, b in zip(xi, xj))
        if not any(sum((2 * F(zk) - a - b) ** 2 for zk, a, b in zip(X[k], xi, xj)) < dd
                   for k in range(n) if k not in (i, j)):
            out.append((i, j))
    return out


def _sqrt_lt_sqrt_minus(a, b, c):
    """Exactly decide sqrt(a) < sqrt(b) - c for rationals a, b >= 0 and c >= 0."""
    # sqrt(a) + c < sqrt(b)  <=>  a + c^2 + 2c sqrt(a) < b
    lhs_rat = a + c * c
    if c == 0:
        return a < b
    if lhs_rat >= b:
        return False
    # 2c sqrt(a) < b - a - c^2 (both sides >= 0)  <=>  4 c^2 a < (b - a - c^2)^2
    return 4 * c * c * a < (b - lhs_rat) ** 2


def grng(P, r, metric):
    """Edges (i<j) of the GRNG of pivots P with radii r by its definition.

    p_k blocks (p_i, p_j) iff d(p_k,p_i) < d(p_i,p_j) - (2 r_i + r_j) and
    d(p_k,p_j) < d(p_i,p_j) - (r_i + 2 r_j)."""
    m = len(P)
    r = [F(x) for x in r]
    K = [[key(P[i], P[j], metric) for j in range(m)] for i in range(m)]

    def lt(kk, kij, c):  # d_k < d_ij - c, with d = sqrt(key) for L2, key for L1
        if metric == L1:
            return kk < kij - c
        return _sqrt_lt_sqrt_minus(kk, kij, c)

    out = []
    for i, j in combinations(range(m), 2):
        c1 = 2 * r[i] + r[j]
        c2 = r[i] + 2 * r[j]
        blocked = any(lt(K[k][i], K[i][j], c1) and lt(K[k][j], K[i][j], c2)
                      for k in range(m) if k not in (i, j))
        if not blocked:
            out.append((i, j))
    return out
