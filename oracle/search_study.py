"""Distance computations per query of the paper's staged RNG search (Algorithm 1 without
Stage VII: Theorem 1, the virtual-pivot prunes of Stages II and III, pivots and members as
interceptors), on the host, as the index grows (oracle only).

The paper reports the search as logarithmic in the index size on uniform low-dimensional data.
Each row: an index of n points with about sqrt(n) * 2 pivots drawn uniformly, 64 queries of the
same generator; the counts exclude the index's own construction.

    python -m oracle.search_study            # prints a markdown table
"""
import numpy as np

from . import L2, rng_search, rng_search_guided


def _points(kind, n, rng):
    if kind == "uniform 2-D":
        return rng.random((n, 2)).astype(np.float32)
    if kind == "uniform 4-D":
        return rng.random((n, 4)).astype(np.float32)
    from paper_2208_10022_gb300 import workloads as wl  # generators only: no method arithmetic
    return wl.gen_points("lin96", n, int(rng.integers(1 << 30)))


def main():
    print("| data | index points | pivots | distances per query | after Stage I | after Stage II | after Stage III "
          "| equal to the definition |")
    print("|---|---:|---:|---:|---:|---:|---:|---|")
    rng = np.random.default_rng(7)
    for kind, sizes in (("uniform 2-D", (2000, 8000, 32000)), ("uniform 4-D", (2000, 8000, 32000)),
                        ("lin96", (2000, 8000, 32000))):
        for n in sizes:
            allp = _points(kind, n + 64, rng)
            X, Q = allp[:n], allp[n:]
            m = int(2 * np.sqrt(n))
            piv = np.sort(rng.choice(n, m, replace=False)).astype(np.int32)
            got, st = rng_search_guided(X, piv, Q, L2)
            want = rng_search(X, Q[:8], L2)
            same = all(np.array_equal(got[j], want[j]) for j in range(8))
            q = len(Q)
            print(f"| {kind} | {n:,} | {m} | {st['distances'] / q:,.0f} | {st['after_stage1'] / q:,.0f} | "
                  f"{st['after_stage2'] / q:,.0f} | {st['after_stage3'] / q:,.0f} | {'8 of 8 checked' if same else 'NO'} |")


if __name__ == "__main__":
    main()
