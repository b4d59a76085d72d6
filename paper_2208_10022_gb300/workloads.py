"""Seeded synthetic workloads shaped like the paper's construction experiments.

This module holds generators only: random coordinates and random nested pivot
index sets.  It contains none of the method's arithmetic, so both the CUDA path's
tests and the CPU oracle can draw their inputs from it.

The paper measures construction on uniform 2-6-D data (Tables 1-3) and on three
real datasets (Table 4: Corel, an MNIST embedding, LA) that are not available
here.  These generators stand in for them:

  uniform8   N x 8  i.i.d. U[0,1)                                       (config "plain")
  mix16      N x 16 mixture of 64 isotropic Gaussians, centres U[0,10]^16,
             sigma 0.5, equal weights                                    (config "at scale")
  lin96      N x 96, intrinsic dimension 8:  x = A z + 0.01 eps,
             z ~ N(0, I_8), A_ij ~ N(0, 1/8), eps ~ N(0, I_96)           (config "precision")
  lin128     N x 128, intrinsic dimension 12: A_ij ~ N(0, 1/12)          (config "learned")

Pivots of each layer are drawn uniformly without replacement; the finest layer
from all points and every coarser layer from the next finer layer, so that coarse
pivots are also fine pivots (as the proof of Theorem 2 requires).
"""
from __future__ import annotations

import dataclasses

import numpy as np

L2, L1 = 0, 1


@dataclasses.dataclass
class Workload:
    name: str
    X: np.ndarray            # float32 [N, D], row-major
    layers: list             # list of int32 pivot-index arrays, coarsest first
    metric: int = L2

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def dim(self) -> int:
        return int(self.X.shape[1])


# name -> (N, D, layer sizes coarsest first, data seed, pivot seed)
SPECS = {
    "uniform8": (1_000, 8, [32], 1000, 2000),
    "mix16": (100_000, 16, [256, 4096], 1001, 2001),
    "lin96": (1_000_000, 96, [1024, 16384, 131072], 1002, 2002),
    "lin128": (2_000_000, 128, [2048, 32768, 262144], 1003, 2003),
}


def gen_points(kind: str, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    if kind == "uniform8":
        return rng.random((n, 8), dtype=np.float64).astype(np.float32)
    if kind == "mix16":
        centres = rng.uniform(0.0, 10.0, size=(64, 16))
        lab = rng.integers(0, 64, size=n)
        x = centres[lab] + 0.5 * rng.standard_normal((n, 16))
        return x.astype(np.float32)
    if kind in ("lin96", "lin128"):
        D, d = (96, 8) if kind == "lin96" else (128, 12)
        A = rng.normal(0.0, np.sqrt(1.0 / d), size=(D, d))
        out = np.empty((n, D), dtype=np.float32)
        step = 1 << 17
        for s in range(0, n, step):
            e = min(n, s + step)
            z = rng.standard_normal((e - s, d))
            eps = rng.standard_normal((e - s, D))
            out[s:e] = (z @ A.T + 0.01 * eps).astype(np.float32)
        return out
    raise ValueError(f"unknown workload kind {kind!r}")


def nested_pivots(n: int, sizes, seed: int):
    """Nested uniform pivot sets, coarsest first; finest drawn from range(n)."""
    rng = np.random.default_rng(seed)
    sizes = [int(s) for s in sizes]
    if any(a > b for a, b in zip(sizes, sizes[1:])) or (sizes and sizes[-1] > n):
        raise ValueError("layer sizes must be non-decreasing and at most n")
    layers = [None] * len(sizes)
    pool = np.arange(n, dtype=np.int64)
    for li in range(len(sizes) - 1, -1, -1):
        pick = rng.choice(pool.shape[0], size=sizes[li], replace=False)
        layers[li] = np.sort(pool[pick]).astype(np.int32)
        pool = layers[li].astype(np.int64)
    return layers


def scaled_layer_sizes(kind: str, n: int):
    """Layer sizes of generator `kind` at n points: the full sizes scaled by n / N (at least 2)."""
    N0, _, sizes0, _, _ = SPECS[kind]
    return [max(2, int(round(s * n / N0))) for s in sizes0]


def make(kind: str, n: int | None = None, metric: int = L2, layer_sizes=None,
         data_seed: int | None = None, pivot_seed: int | None = None) -> Workload:
    """A workload of generator `kind`; with n smaller than the full size, the layer
    sizes scale in proportion (at least 2 pivots per layer)."""
    N0, _, sizes0, ds, ps = SPECS[kind]
    n = N0 if n is None else int(n)
    if layer_sizes is None:
        layer_sizes = scaled_layer_sizes(kind, n)
    X = gen_points(kind, n, ds if data_seed is None else data_seed)
    layers = nested_pivots(n, layer_sizes, ps if pivot_seed is None else pivot_seed)
    return Workload(name=f"{kind}-{n}", X=X, layers=layers, metric=metric)


def subsample(w: Workload, n_sub: int, seed: int) -> Workload:
    """Seeded subsample of a workload's points with its own nested pivots, the layer
    sizes scaled by n_sub / n (the subsample's RNG is its own, not a restriction)."""
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(w.n, size=n_sub, replace=False))
    X = np.ascontiguousarray(w.X[idx])
    sizes = [max(2, int(round(len(l) * n_sub / w.n))) for l in w.layers]
    layers = nested_pivots(n_sub, sizes, seed + 1)
    return Workload(name=f"{w.name}-sub{n_sub}", X=X, layers=layers, metric=w.metric)


def insertion_batches(n_batches: int, seed: int = 4000, lo: int = 1000, hi: int = 65536):
    """Batch sizes floor(exp(U[ln lo, ln hi])) for incremental insertion."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_batches))).astype(np.int64)
