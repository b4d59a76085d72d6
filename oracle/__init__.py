"""ctypes binding of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()``, the CPU-baseline legs of ``bench.py`` and the
oracle's own host studies (``python -m oracle.pivoting_study``, ``python -m oracle.search_study``)
import this package.  The product library never does.
"""
import ctypes
import os

import numpy as np

from . import build as _build

L2, L1 = 0, 1
_lib = None


def use_library(path):
    """Bind this module to another build of the oracle (used to check that the pins
    catch deliberately broken builds)."""
    global _lib, _path
    _lib, _path = None, path


_path = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_path or _build.build())
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        _lib.orc_key.restype = f64
        _lib.orc_key.argtypes = [P, P, i32, i32]
        _lib.orc_dist.restype = f64
        _lib.orc_dist.argtypes = [P, P, i32, i32]
        _lib.orc_rng_brute.restype = i64
        _lib.orc_rng_brute.argtypes = [P, i64, i32, i32, P, i64]
        _lib.orc_rng_row.restype = i64
        _lib.orc_rng_row.argtypes = [P, i64, i32, i32, i64, P, i64]
        _lib.orc_rng_rows.restype = i32
        _lib.orc_rng_rows.argtypes = [P, i64, i32, i32, P, i64, P, i64, P]
        _lib.orc_rng_search.restype = i32
        _lib.orc_beta_brute.restype = i64
        _lib.orc_grng_insert_pivot.restype = i32
        _lib.orc_grng_insert_pivot.argtypes = [P, P, i64, i32, i32, P, P, P]
        _lib.orc_beta_brute.argtypes = [P, i64, i32, ctypes.c_double, P, i64]
        _lib.orc_rng_search.argtypes = [P, i64, P, i64, i32, i32, P, i64, P]
        _lib.orc_verify_witness.restype = i32
        _lib.orc_verify_witness.argtypes = [P, i32, i32, i64, i64, i64]
        _lib.orc_set_threads.restype = i32
        _lib.orc_set_threads.argtypes = [i32]
        _lib.orc_max_threads.restype = i32
        _lib.orc_max_threads.argtypes = []
        if hasattr(_lib, "orc_rng_guided"):  # absent from single-file builds of the pin tests
            _lib.orc_rng_guided.restype = i64
            _lib.orc_rng_guided.argtypes = [P, i64, i32, i32, P, P, i32, P, i64, P]
            _lib.orc_candidates_rules.restype = i32
            _lib.orc_rng_search_guided.restype = i32
            _lib.orc_rng_search_guided.argtypes = [P, i64, i32, i32, P, i32, P, i64, P, i64, P, P]
            _lib.orc_candidates_rules.argtypes = [P, i64, i32, i32, P, i32, ctypes.c_double, i32, P, P, P]
        _lib.orc_emst.restype = i64
        _lib.orc_emst.argtypes = [P, i64, i32, i32, P]
        _lib.orc_grng_brute.restype = i64
        _lib.orc_grng_brute.argtypes = [P, P, i64, i32, i32, P, i64]
        _lib.orc_grng_row.restype = i64
        _lib.orc_grng_row.argtypes = [P, P, i64, i32, i32, i64, P, i64]
        _lib.orc_assign.restype = i32
        _lib.orc_assign.argtypes = [P, i32, i32, P, i64, P, P, i32, P, P, P, P]
        if hasattr(_lib, "orc_mlp_forward"):
            _lib.orc_mlp_nparams.restype = i64
            _lib.orc_mlp_nparams.argtypes = []
            _lib.orc_mlp_forward.restype = None
            _lib.orc_mlp_forward.argtypes = [P, P, i64, P]
            _lib.orc_mlp_backward.restype = f64
            _lib.orc_mlp_backward.argtypes = [P, P, P, P, i64, P]
    return _lib


def _f32(X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    assert X.ndim == 2
    return X


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(t):
    """Use t OpenMP threads from now on; returns the previous count."""
    return int(lib().orc_set_threads(int(t)))


def max_threads():
    return int(lib().orc_max_threads())


def key(a, b, metric=L2):
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return lib().orc_key(_p(a), _p(b), a.shape[0], metric)


def dist(a, b, metric=L2):
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return lib().orc_dist(_p(a), _p(b), a.shape[0], metric)


def _edges_call(fn, *args):
    cnt = fn(*args, None, 0)
    if cnt < 0:
        raise MemoryError("oracle allocation failed")
    out = np.zeros((max(cnt, 1), 2), dtype=np.int32)
    cnt2 = fn(*args, _p(out), cnt)
    assert cnt2 == cnt
    return out[:cnt]


def rng_brute(X, metric=L2):
    """RNG of X by Eq. 1 over all triples: sorted (i<j) int32 edges [E,2]."""
    X = _f32(X)
    return _edges_call(lib().orc_rng_brute, _p(X), X.shape[0], X.shape[1], metric)


def rng_row(X, x, metric=L2):
    """Exact RNG neighbours of point x (ascending int32 array)."""
    X = _f32(X)
    n = X.shape[0]
    out = np.zeros(max(n, 1), dtype=np.int32)
    cnt = lib().orc_rng_row(_p(X), n, X.shape[1], metric, int(x), _p(out), n)
    if cnt < 0:
        raise MemoryError("oracle allocation failed")
    return out[:cnt]


def rng_rows(X, xs, metric=L2, row_cap=4096):
    """Exact RNG neighbourhoods of the points xs (a list of ascending int32 arrays), the
    rows spread over the host's cores."""
    X = _f32(X)
    xs = np.ascontiguousarray(xs, dtype=np.int64)
    nb = np.zeros((max(len(xs), 1), row_cap), np.int32)
    cnt = np.zeros(max(len(xs), 1), np.int64)
    rc = lib().orc_rng_rows(_p(X), X.shape[0], X.shape[1], metric, _p(xs), len(xs), _p(nb), row_cap, _p(cnt))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    if len(xs) and cnt.max() > row_cap:
        raise ValueError("a neighbourhood exceeds row_cap")
    return [nb[t, :cnt[t]].copy() for t in range(len(xs))]


def rng_search(X, Q, metric=L2, row_cap=4096):
    """RNG search (Sec. 2, Algorithm 1 without Stage VII): for each query row of Q, its
    RNG neighbours among the index points X (a list of ascending int32 arrays).  A query
    does not join the index: only index points block, never another query."""
    X = _f32(X)
    Q = _f32(Q)
    if Q.shape[1] != X.shape[1]:
        raise ValueError("queries and index differ in dimension")
    m = Q.shape[0]
    nb = np.zeros((max(m, 1), row_cap), np.int32)
    cnt = np.zeros(max(m, 1), np.int64)
    rc = lib().orc_rng_search(_p(X), X.shape[0], _p(Q), m, X.shape[1], metric, _p(nb), row_cap, _p(cnt))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    if m and cnt.max() > row_cap:
        raise ValueError("a neighbourhood exceeds row_cap")
    return [nb[t, :cnt[t]].copy() for t in range(m)]


def beta_skeleton(X, beta):
    """Lune-based beta-skeleton of X for 1 <= beta <= 2 (L2; beta = 1 the Gabriel graph, 2 the
    RNG), all triples: sorted (i<j) int32 edges [E,2]."""
    X = _f32(X)
    fn = lib().orc_beta_brute
    args = (_p(X), X.shape[0], X.shape[1], float(beta))
    cnt = fn(*args, None, 0)
    if cnt == -2:
        raise ValueError("beta must lie in [1, 2]")
    if cnt < 0:
        raise MemoryError("oracle allocation failed")
    out = np.zeros((max(cnt, 1), 2), dtype=np.int32)
    assert fn(*args, _p(out), cnt) == cnt
    return out[:cnt]


def rng_guided(X, layers, metric=L2, with_stats=False):
    """RNG of X by the paper's pivot-guided method (Secs. 2-3: layers, GRNGs under Theorem 2,
    exemplar pairs under Theorem 1, Stages IV and VI), FP64 on the host: sorted edges [E, 2]
    and, with with_stats, (distance computations, candidate pairs, Stage VI member tests)."""
    X = _f32(X)
    piv = np.ascontiguousarray(np.concatenate([np.asarray(l, np.int32) for l in layers]), dtype=np.int32)
    ms = np.ascontiguousarray([len(l) for l in layers], dtype=np.int32)
    st = np.zeros(3, np.int64)
    args = (_p(X), X.shape[0], X.shape[1], metric, _p(piv), _p(ms), len(layers))
    cnt = lib().orc_rng_guided(*args, None, 0, _p(st))
    if cnt < 0:
        raise MemoryError("oracle allocation failed")
    out = np.zeros((max(cnt, 1), 2), dtype=np.int32)
    cnt2 = lib().orc_rng_guided(*args, _p(out), cnt, _p(st))
    assert cnt2 == cnt
    return (out[:cnt], tuple(int(v) for v in st)) if with_stats else out[:cnt]


def rng_search_guided(X, piv, Q, metric=L2, row_cap=4096):
    """RNG search by the paper's Stages I-VI over one pivot layer (Algorithm 1 without Stage
    VII): (list of ascending int32 neighbour arrays per query, {"distances": computations,
    "after_stage1"/"after_stage2"/"after_stage3": exemplars left, summed over the queries})."""
    X = _f32(X)
    Q = _f32(Q)
    piv = np.ascontiguousarray(piv, dtype=np.int32)
    m = Q.shape[0]
    nb = np.zeros((max(m, 1), row_cap), np.int32)
    cnt = np.zeros(max(m, 1), np.int64)
    st = np.zeros(4, np.int64)
    rc = lib().orc_rng_search_guided(_p(X), X.shape[0], X.shape[1], metric, _p(piv), len(piv), _p(Q), m,
                                     _p(nb), row_cap, _p(cnt), _p(st))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    if m and cnt.max() > row_cap:
        raise ValueError("a neighbourhood exceeds row_cap")
    return ([nb[t, :cnt[t]].copy() for t in range(m)],
            {"distances": int(st[0]), "after_stage1": int(st[1]), "after_stage2": int(st[2]),
             "after_stage3": int(st[3])})


def candidate_rules(X, piv, r, metric=L2, want_sets=False, promote=False):
    """Stage I candidate pairs of one pivot layer under the nearest-pivot rule with per-pivot
    radii (A) and under the uniform radius r with every pivot within r a parent (B), each with
    its own GRNG (Sec. 2, Theorem 1); promote makes every point with no pivot within r a pivot
    under B first.  {"a": count, "b": count, "no_parent": points, "memberships": parent links
    under B, "pivots_b": B's pivots, "a_on_b_pivots": rule A's count on B's pivots}; with want_sets
    also the candidate sets of pairs i < j."""
    X = _f32(X)
    piv = np.ascontiguousarray(piv, dtype=np.int32)
    n = X.shape[0]
    st = np.zeros(6, np.int64)
    ca = np.zeros((n, n), np.uint8) if want_sets else None
    cb = np.zeros((n, n), np.uint8) if want_sets else None
    rc = lib().orc_candidates_rules(_p(X), n, X.shape[1], metric, _p(piv), len(piv), float(r), int(promote),
                                    _p(ca) if want_sets else None, _p(cb) if want_sets else None, _p(st))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    out = {"a": int(st[0]), "b": int(st[1]), "no_parent": int(st[2]), "memberships": int(st[3]),
           "pivots_b": int(st[4]), "a_on_b_pivots": int(st[5])}
    if want_sets:
        out["set_a"] = {(int(i), int(j)) for i, j in zip(*np.nonzero(np.triu(ca, 1)))}
        out["set_b"] = {(int(i), int(j)) for i, j in zip(*np.nonzero(np.triu(cb, 1)))}
    return out


def verify_witness(X, x, y, z, metric=L2):
    """True when z (not x or y) lies strictly inside the lune of (x, y) (Eq. 1)."""
    X = _f32(X)
    return bool(lib().orc_verify_witness(_p(X), X.shape[1], metric, int(x), int(y), int(z)))


def emst(X, metric=L2):
    """A minimum spanning tree of the complete graph (Prim, canonical keys): int32 [n-1, 2]."""
    X = _f32(X)
    n = X.shape[0]
    out = np.zeros((max(n - 1, 1), 2), np.int32)
    cnt = lib().orc_emst(_p(X), n, X.shape[1], metric, _p(out))
    if cnt < 0:
        raise MemoryError("oracle allocation failed")
    return out[:cnt]


def grng_brute(P, r, metric=L2):
    """GRNG of pivots P[m,D] with radii r[m] by its definition: sorted edges [E,2]."""
    P = _f32(P)
    r = np.ascontiguousarray(r, dtype=np.float64)
    return _edges_call(lib().orc_grng_brute, _p(P), _p(r), P.shape[0], P.shape[1], metric)


def grng_row(P, r, i, metric=L2):
    P = _f32(P)
    r = np.ascontiguousarray(r, dtype=np.float64)
    m = P.shape[0]
    out = np.zeros(max(m, 1), dtype=np.int32)
    cnt = lib().orc_grng_row(_p(P), _p(r), m, P.shape[1], metric, int(i), _p(out), m)
    if cnt < 0:
        raise MemoryError("oracle allocation failed")
    return out[:cnt]


def grng_insert_pivot(P, r, edges, metric=L2):
    """GRNG after a new pivot joins (Stage VII): P[m+1, D] with the new pivot last, r[m+1],
    edges = the GRNG of the first m (pairs i < j).  Returns (sorted edges [E, 2] of all m+1,
    (old links tested, old links removed, links of the new pivot))."""
    P = _f32(P)
    r = np.ascontiguousarray(r, dtype=np.float64)
    m = P.shape[0] - 1
    links = np.zeros((max(m, 1), max(m, 1)), np.uint8)
    for i, j in np.asarray(edges, dtype=np.int64).reshape(-1, 2):
        links[min(i, j), max(i, j)] = 1
    out = np.zeros((m + 1, m + 1), np.uint8)
    st = np.zeros(3, np.int64)
    if lib().orc_grng_insert_pivot(_p(P), _p(r), m, P.shape[1], metric, _p(links), _p(out), _p(st)) != 0:
        raise MemoryError("oracle allocation failed")
    E = np.argwhere(np.triu(out, 1)).astype(np.int32)
    return E, tuple(int(v) for v in st)


def assign(X, members, pivots, member_r=None, metric=L2):
    """Nearest-pivot assignment, distances, radii and delta_max of one layer."""
    X = _f32(X)
    members = np.ascontiguousarray(members, dtype=np.int32)
    pivots = np.ascontiguousarray(pivots, dtype=np.int32)
    nm, m = members.shape[0], pivots.shape[0]
    a = np.zeros(max(nm, 1), np.int32)
    d = np.zeros(max(nm, 1), np.float64)
    r = np.zeros(max(m, 1), np.float64)
    dm = np.zeros(max(m, 1), np.float64)
    mr = None if member_r is None else np.ascontiguousarray(member_r, dtype=np.float64)
    rc = lib().orc_assign(_p(X), X.shape[1], metric, _p(members), nm,
                          None if mr is None else _p(mr), _p(pivots), m, _p(a), _p(d), _p(r), _p(dm))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return a[:nm], d[:nm], r[:m], dm[:m]


def build_layers(X, layers, metric=L2):
    """Assignment/radii for a nested hierarchy, finest first (Eq. 2; Sec. 3).

    layers: list of pivot-index arrays, coarsest first.  Returns a list (coarsest
    first) of dicts with keys pivots, assign, dist, radius, delta_max.
    """
    n = X.shape[0]
    out = [None] * len(layers)
    members = np.arange(n, dtype=np.int32)
    member_r = None
    for li in range(len(layers) - 1, -1, -1):
        piv = np.asarray(layers[li], dtype=np.int32)
        a, d, r, dm = assign(X, members, piv, member_r, metric)
        out[li] = dict(pivots=piv, assign=a, dist=d, radius=r, delta_max=dm)
        members, member_r = piv, r
    return out


# ---- interceptor-ranking network (extension of Stage V) ---------------------------------
MLP_IN, MLP_H = 32, 128


def mlp_nparams():
    return int(lib().orc_mlp_nparams())


def mlp_forward(params, X):
    """FP64 logits of the samples X[N][32] under the parameter vector `params`."""
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, MLP_IN)
    out = np.zeros(X.shape[0], np.float64)
    lib().orc_mlp_forward(_p(P), _p(X), X.shape[0], _p(out))
    return out


def mlp_loss_grad(params, X, y, w=None):
    """(loss, gradient) of the weighted mean logistic loss, FP64."""
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, MLP_IN)
    y = np.ascontiguousarray(y, dtype=np.float64)
    wv = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    g = np.zeros(P.shape[0], np.float64)
    loss = lib().orc_mlp_backward(_p(P), _p(X), _p(y), None if wv is None else _p(wv), X.shape[0], _p(g))
    return float(loss), g
