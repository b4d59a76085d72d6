"""Stage I candidate pairs under two pivot-membership rules, on the host (oracle only).

Rule A: every point joins its nearest pivot, whose radius is its largest member distance.
Rule B: the paper's uniform radius r; every pivot within r of a point is a parent of it, and a
point with no pivot within r becomes a pivot itself (Sec. 2).  Under each rule a pair stays a
candidate only when its parents are equal or GRNG-linked (Theorem 1; under B, every parent
pair).  The table compares the two at the same pivot sets (rule A run on B's pivots too).

    python -m oracle.pivoting_study            # prints a markdown table
"""
import numpy as np

from . import candidate_rules, dist, L2


def _row(name, X, piv, scale):
    n = X.shape[0]
    nn = np.array([min(dist(X[i], X[p], L2) for p in piv) for i in range(n)])
    r = float(np.median(nn) * scale) if scale else float(nn.max())
    res = candidate_rules(X, piv, r, L2, promote=True)
    pairs = n * (n - 1) // 2
    return (f"| {name} | {len(piv)} | {'covering' if not scale else f'{scale:g} x median'} ({r:.4g}) | "
            f"{res['pivots_b']} | {res['memberships'] / n:.2f} | {res['b'] / pairs:.3f} | "
            f"{res['a_on_b_pivots'] / pairs:.3f} | {res['a'] / pairs:.3f} |")


def main():
    print("| points | pivots given | r | pivots under B | parents per point (B) | candidates B | "
          "candidates A, B's pivots | candidates A, given pivots |")
    print("|---|---:|---|---:|---:|---:|---:|---:|")
    rng = np.random.default_rng(5)
    for d in (2, 4):
        X = rng.random((3000, d)).astype(np.float32)
        piv = np.sort(rng.choice(3000, 150, replace=False)).astype(np.int32)
        for scale in (0, 2.0, 1.0):
            print(_row(f"uniform {d}-D, 3,000", X, piv, scale))
    from paper_2208_10022_gb300 import workloads as wl  # generators only: no method arithmetic
    w = wl.make("mix16", n=3000)
    for scale in (0, 1.0):
        print(_row("mix16, 3,000", w.X, w.layers[-1], scale))


if __name__ == "__main__":
    main()
