"""Python binding of libgrng (include/grng.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module converts numpy
arrays / torch tensors into pointers and statuses into exceptions.  There is no
fallback: if the compiled library is absent, importing the binding's functions
raises.

    import paper_2208_10022_gb300 as grng
    ix = grng.Index(points, n_layers=2)            # float32 [n, dim], host or cuda
    ix.build_layer(1, fine_pivots); ix.build_layer(0, coarse_pivots)
    ix.link_pivots(0); ix.link_pivots(1)
    ix.rng_build_exact()
    edges = ix.rng_edges()                          # int32 [E, 2], i < j, sorted
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgrng.so")

GRNG_OK, GRNG_EINVAL, GRNG_ENOMEM, GRNG_ECUDA, GRNG_ETIMEOUT, GRNG_ETRUNC = 0, 1, 2, 3, 4, 5
GRNG_EINTERNAL, GRNG_ESTATE, GRNG_ENOTIMPL = 6, 7, 8
L2, L1 = 0, 1
FP32, BF16, FP8 = 0, 1, 2

EXPORTS = [
    "grng_default_opts", "grng_create", "grng_build_layer", "grng_link_pivots", "grng_adjacency_rows",
    "rng_build_exact", "rng_build_skeleton", "rng_insert_batch", "rng_search_batch", "rng_search_result",
    "rng_edges", "grng_stats", "grng_destroy", "grng_last_error",
]


class GrngError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"grng status {status}: {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [
        ("metric", ctypes.c_int32), ("precision", ctypes.c_int32), ("n_layers", ctypes.c_int32),
        ("knn_k", ctypes.c_int32), ("k_shortlist", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("mlp_weights", ctypes.c_void_p), ("mlp_bytes", ctypes.c_size_t), ("spin_limit", ctypes.c_int64),
        ("cuda_stream", ctypes.c_void_p), ("flags", ctypes.c_uint64),
    ]


_lib = None


def lib():
    """The loaded C library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libgrng.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        L.grng_default_opts.argtypes = [ctypes.POINTER(Opts)]
        L.grng_default_opts.restype = None
        L.grng_create.argtypes = [ctypes.POINTER(P), P, i64, i32, ctypes.POINTER(Opts)]
        L.grng_build_layer.argtypes = [P, i32, P, i32, P, P, P]
        L.grng_link_pivots.argtypes = [P, i32, P, P, P, i64, ctypes.POINTER(i64)]
        L.grng_adjacency_rows.argtypes = [P, i32, i64, i64, P, P, i64, ctypes.POINTER(i64)]
        L.rng_build_exact.argtypes = [P]
        L.rng_build_skeleton.argtypes = [P, ctypes.c_double]
        L.rng_insert_batch.argtypes = [P, P, i64]
        L.rng_search_batch.argtypes = [P, P, i64, ctypes.POINTER(i64)]
        L.rng_search_result.argtypes = [P, P, P, i64]
        L.rng_edges.argtypes = [P, P, i64, ctypes.POINTER(i64)]
        L.grng_stats.argtypes = [P, ctypes.c_char_p, sz]
        L.grng_destroy.argtypes = [P]
        L.grng_destroy.restype = None
        L.grng_last_error.argtypes = []
        L.grng_last_error.restype = ctypes.c_char_p
        f32p = ctypes.POINTER(ctypes.c_float)
        L.grng_mlp_nparams.argtypes = []
        L.grng_mlp_nparams.restype = i64
        L.grng_mlp_score.argtypes = [P, P, i64, P]
        L.grng_mlp_loss_grad.argtypes = [P, P, P, P, i64, f32p, P]
        L.grng_mlp_train.argtypes = [P, P, P, i64, i32, i32, ctypes.c_float, P, f32p]
        L.grng_mlp_dataset.argtypes = [P, P, P, i64, ctypes.POINTER(i64)]
        L.grng_tc_keys.argtypes = [P, i64, i32, P]
        for f in ("grng_create", "grng_build_layer", "grng_link_pivots", "grng_adjacency_rows",
                  "rng_build_exact", "rng_build_skeleton", "rng_insert_batch", "rng_search_batch",
                  "rng_search_result", "rng_edges",
                  "grng_stats", "grng_mlp_score",
                  "grng_mlp_loss_grad", "grng_mlp_train", "grng_mlp_dataset", "grng_tc_keys"):
            getattr(L, f).restype = i32
        _lib = L
    return _lib


def _check(st):
    if st != GRNG_OK:
        raise GrngError(st, lib().grng_last_error().decode())


def _ptr(a):
    """Pointer of a numpy array or torch tensor (host or device); keeps no reference."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch.Tensor


def _contig(a, dtype):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=dtype)
    import torch
    tdt = {np.float32: torch.float32, np.int32: torch.int32, np.float64: torch.float64}[dtype]
    return a.to(tdt).contiguous()


class Index:
    """An index over a point set (owns the library's grng_index)."""

    def __init__(self, points, n_layers=1, metric=L2, precision=FP32, knn_k=32, stream=None, flags=0,
                 mlp_params=None, k_shortlist=0, spin_limit=0):
        self._h = ctypes.c_void_p()
        pts = _contig(points, np.float32)
        n, dim = int(pts.shape[0]), int(pts.shape[1])
        o = Opts()
        lib().grng_default_opts(ctypes.byref(o))
        o.metric, o.precision, o.n_layers, o.knn_k, o.flags = metric, precision, n_layers, knn_k, flags
        o.spin_limit = spin_limit
        if mlp_params is not None:
            w = _contig(mlp_params, np.float32)
            o.mlp_weights, o.mlp_bytes, o.k_shortlist = _ptr(w), 4 * int(w.shape[0]), k_shortlist
        if stream is not None:
            o.cuda_stream = stream if isinstance(stream, int) else stream.cuda_stream
        _check(lib().grng_create(ctypes.byref(self._h), _ptr(pts), n, dim, ctypes.byref(o)))
        self.n, self.dim, self.n_layers, self.metric = n, dim, n_layers, metric
        self._m = [0] * n_layers

    def close(self):
        if self._h:
            lib().grng_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_layer(self, layer, pivot_idx, outputs=True):
        """Assignment, radii and delta_max of one layer (copied to numpy if outputs)."""
        piv = _contig(pivot_idx, np.int32)
        m = int(piv.shape[0])
        if not outputs:
            _check(lib().grng_build_layer(self._h, layer, _ptr(piv), m, None, None, None))
            self._m[layer] = m
            return None
        n_mem = self.n if layer == self.n_layers - 1 else self._m[layer + 1]
        assign = np.zeros(max(n_mem, 1), np.int32)
        radius = np.zeros(max(m, 1), np.float64)
        delta = np.zeros(max(m, 1), np.float64)
        _check(lib().grng_build_layer(self._h, layer, _ptr(piv), m, assign.ctypes.data, radius.ctypes.data,
                                      delta.ctypes.data))
        self._m[layer] = m
        return assign[:n_mem], radius[:m], delta[:m]

    def link_pivots(self, layer, radius_override=None, want_adjacency=True):
        """GRNG of one layer; returns (off, adj) in pivot order, or None."""
        m = self._m[layer]
        r = None if radius_override is None else _contig(radius_override, np.float64)
        if r is None:
            _check(lib().grng_link_pivots(self._h, layer, None, None, None, 0, None))
            return self.adjacency_rows(layer, 0, m) if want_adjacency else None
        off = np.zeros(m + 1, np.int64)
        need = ctypes.c_int64(0)
        cap = m * (m - 1) if m <= 4096 else 0
        adj = np.zeros(max(cap, 1), np.int32)
        st = lib().grng_link_pivots(self._h, layer, _ptr(r), off.ctypes.data, adj.ctypes.data, cap,
                                    ctypes.byref(need))
        if st == GRNG_ETRUNC:  # the override graph is not stored: compute again with room
            adj = np.zeros(max(need.value, 1), np.int32)
            st = lib().grng_link_pivots(self._h, layer, _ptr(r), off.ctypes.data, adj.ctypes.data, need.value,
                                        ctypes.byref(need))
        _check(st)
        return off, adj[:need.value]

    def adjacency_rows(self, layer, r0, r1):
        off = np.zeros(r1 - r0 + 1, np.int64)
        need = ctypes.c_int64(0)
        _check(lib().grng_adjacency_rows(self._h, layer, r0, r1, off.ctypes.data, None, 0, ctypes.byref(need)))
        adj = np.zeros(max(need.value, 1), np.int32)
        _check(lib().grng_adjacency_rows(self._h, layer, r0, r1, off.ctypes.data, adj.ctypes.data, need.value,
                                         ctypes.byref(need)))
        return off, adj[:need.value]

    def rng_build_exact(self):
        _check(lib().rng_build_exact(self._h))

    def rng_build_skeleton(self, beta):
        """Lune-based beta-skeleton (1 <= beta <= 2, L2) as the stored graph; read it with rng_edges."""
        _check(lib().rng_build_skeleton(self._h, float(beta)))

    def rng_insert_batch(self, points):
        pts = _contig(points, np.float32)
        _check(lib().rng_insert_batch(self._h, _ptr(pts), int(pts.shape[0])))

    def rng_search_batch(self, queries):
        """Search m queries [m, dim] (host or cuda); returns the number of (query, neighbour)
        pairs, kept in the index for rng_search_result."""
        q = _contig(queries, np.float32)
        tot = ctypes.c_int64(0)
        _check(lib().rng_search_batch(self._h, _ptr(q), int(q.shape[0]), ctypes.byref(tot)))
        self._search_m = int(q.shape[0])
        return tot.value

    def rng_search_result(self, off=None, nbrs=None):
        """(off int64 [m+1], nbrs int32 [off[m]]) of the last search; `off`/`nbrs` may be
        preallocated numpy arrays or cuda tensors of at least that size."""
        if off is None:
            off = np.zeros(getattr(self, "_search_m", 0) + 1, np.int64)
        _check(lib().rng_search_result(self._h, _ptr(off), None, 0))
        total = int(off[-1]) if isinstance(off, np.ndarray) else int(off[-1].item())
        if nbrs is None:
            nbrs = np.zeros(max(total, 1), np.int32)
        _check(lib().rng_search_result(self._h, _ptr(off), _ptr(nbrs), total))
        return off, nbrs[:total]

    def rng_search(self, queries):
        """Neighbours of each query among the index points: a list of ascending int32 arrays."""
        self.rng_search_batch(queries)
        off, nb = self.rng_search_result()
        return [nb[off[j]:off[j + 1]] for j in range(len(off) - 1)]

    def n_edges(self):
        ne = ctypes.c_int64(0)
        _check(lib().rng_edges(self._h, None, 0, ctypes.byref(ne)))
        return ne.value

    def rng_edges(self, out=None):
        """Edges int32 [E, 2]; `out` may be a preallocated numpy array or cuda tensor."""
        ne = self.n_edges()
        if out is None:
            out = np.zeros((max(ne, 1), 2), np.int32)
        _check(lib().rng_edges(self._h, _ptr(out), ne, None))
        return out[:ne]

    def mlp_dataset(self):
        """(features [N, 32], labels [N]) recorded by the last RNG build (GRNG_FLAG_RECORD_MLP)."""
        cnt = ctypes.c_int64(0)
        _check(lib().grng_mlp_dataset(self._h, None, None, 0, ctypes.byref(cnt)))
        n = cnt.value
        F = np.zeros((max(n, 1), MLP_IN), np.float32)
        y = np.zeros(max(n, 1), np.float32)
        _check(lib().grng_mlp_dataset(self._h, F.ctypes.data, y.ctypes.data, n, ctypes.byref(cnt)))
        return F[:n], y[:n]

    def stats(self):
        buf = ctypes.create_string_buffer(1 << 16)
        _check(lib().grng_stats(self._h, buf, len(buf)))
        return json.loads(buf.value.decode())


GRNG_FLAG_SHORT_LISTS = 1
GRNG_FLAG_RECORD_MLP = 2
GRNG_FLAG_SMALL_BUFFERS = 4
MLP_IN = 32


def tc_keys(points):
    """Tensor-core (split BF16) Gram keys of all pairs of at most 256 points, float32 [n, n]."""
    X = np.ascontiguousarray(points, np.float32)
    n, d = X.shape
    out = np.zeros((n, n), np.float32)
    _check(lib().grng_tc_keys(X.ctypes.data, n, d, out.ctypes.data))
    return out


def mlp_nparams():
    return int(lib().grng_mlp_nparams())


def mlp_score(params, feats):
    """Logits of feats [N, 32] (BF16 weights, FP32 accumulation), numpy float32."""
    P = np.ascontiguousarray(params, np.float32)
    F = np.ascontiguousarray(feats, np.float32).reshape(-1, MLP_IN)
    out = np.zeros(F.shape[0], np.float32)
    _check(lib().grng_mlp_score(P.ctypes.data, F.ctypes.data, F.shape[0], out.ctypes.data))
    return out


def mlp_loss_grad(params, feats, labels, weights=None):
    """(loss, gradient) of the weighted mean logistic loss, FP32 on the GPU."""
    P = np.ascontiguousarray(params, np.float32)
    F = np.ascontiguousarray(feats, np.float32).reshape(-1, MLP_IN)
    y = np.ascontiguousarray(labels, np.float32)
    w = None if weights is None else np.ascontiguousarray(weights, np.float32)
    g = np.zeros(P.shape[0], np.float32)
    loss = ctypes.c_float(0.0)
    _check(lib().grng_mlp_loss_grad(P.ctypes.data, F.ctypes.data, y.ctypes.data, None if w is None else w.ctypes.data,
                                    F.shape[0], ctypes.byref(loss), g.ctypes.data))
    return float(loss.value), g


def mlp_train(params, feats, labels, weights=None, epochs=10, batch=4096, lr=1e-3):
    """Adam on the GPU; returns (trained parameters, mean loss of the last pass)."""
    P = np.array(params, np.float32, copy=True)
    F = np.ascontiguousarray(feats, np.float32).reshape(-1, MLP_IN)
    y = np.ascontiguousarray(labels, np.float32)
    w = None if weights is None else np.ascontiguousarray(weights, np.float32)
    loss = ctypes.c_float(0.0)
    _check(lib().grng_mlp_train(F.ctypes.data, y.ctypes.data, None if w is None else w.ctypes.data, F.shape[0],
                                epochs, batch, lr, P.ctypes.data, ctypes.byref(loss)))
    return P, float(loss.value)


def mlp_init(seed=0):
    """He-normal initial parameters (numpy, seeded), biases zero."""
    rng = np.random.default_rng(seed)
    P = np.zeros(mlp_nparams(), np.float32)
    H, I = 128, MLP_IN
    P[:H * I] = rng.normal(0.0, np.sqrt(2.0 / I), H * I)
    o = H * I + H
    P[o:o + H * H] = rng.normal(0.0, np.sqrt(2.0 / H), H * H)
    o += H * H + H
    P[o:o + H] = rng.normal(0.0, np.sqrt(1.0 / H), H)
    return P


def build_all(X, layers, metric=L2, knn_k=32, want_adjacency=False, stream=None, flags=0, precision=FP32,
              mlp_params=None, k_shortlist=0, spin_limit=0):
    """Build every layer (finest first), link every layer (coarsest first) and the RNG."""
    ix = Index(X, n_layers=len(layers), metric=metric, knn_k=knn_k, stream=stream, flags=flags,
               precision=precision, mlp_params=mlp_params, k_shortlist=k_shortlist, spin_limit=spin_limit)
    out = {"layers": [None] * len(layers), "grng": [None] * len(layers)}
    for li in range(len(layers) - 1, -1, -1):
        out["layers"][li] = ix.build_layer(li, layers[li])
    for li in range(len(layers)):
        out["grng"][li] = ix.link_pivots(li, want_adjacency=want_adjacency)
    ix.rng_build_exact()
    out["edges"] = ix.rng_edges()
    return ix, out
