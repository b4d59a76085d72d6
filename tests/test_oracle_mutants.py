"""The pins must catch plausible mistakes planted in a copy of the oracle.

Each mutant is a textual edit of oracle/grng_oracle.c compiled into a temporary
library; the pins run against it in a fresh process and at least one must fail.
The committed oracle is never modified.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "grng_oracle.c")

MUTANTS = {
    "closed_lune": ("if (m < dij) blocked = 1;", "if (m <= dij) blocked = 1;"),
    "lune_min_not_max": ("double m = a > b ? a : b;\n                if (m < dij)",
                         "double m = a < b ? a : b;\n                if (m < dij)"),
    "l2_no_square": ("double sq = t * t;", "double sq = fabs(t);"),
    "l1_signed": ("acc = acc + fabs(t);", "acc = acc + t;"),
    "grng_swapped_radii": ("double t1 = dij - (2.0 * ri + rj);", "double t1 = dij - (ri + 2.0 * rj);"),
    "grng_single_radius": ("double t2 = dij - (ri + 2.0 * rj);", "double t2 = dij - (ri + rj);"),
    "grng_closed": ("return (dki < t1) && (dkj < t2);", "return (dki <= t1) && (dkj <= t2);"),
    "grng_or": ("return (dki < t1) && (dkj < t2);", "return (dki < t1) || (dkj < t2);"),
    "grng_zero_special_dropped": ("if (ri == 0.0 && rj == 0.0) return (kki < kij) && (kkj < kij);", ""),
    "assign_last_tie": ("if (best < 0 || k < bk)", "if (best < 0 || k <= bk)"),
    "radius_without_member_radius": ("double rr = ds[t] + (member_r ? member_r[t] : 0.0);", "double rr = ds[t];"),
    "no_self_assign": ("if (piv[p] == members[t]) { best = p; break; }", ""),
    "row_scan_stops_early": ("if (!(o[q].k < dxy)) break;", "if (!(o[q].k < 0.5 * dxy)) break;"),
    "delta_max_with_member_radius": ("if (delta_max && ds[t] > delta_max[as[t]]) delta_max[as[t]] = ds[t];",
                                     "if (delta_max && rr > delta_max[as[t]]) delta_max[as[t]] = rr;"),
    "witness_closed_lune": ("return m < dxy ? 1 : 0;", "return m <= dxy ? 1 : 0;"),
    "search_closed_lune": ("if (dxz < dqx) blocked = 1;", "if (dxz <= dqx) blocked = 1;"),
    "search_scan_stops_early": ("if (!(o[t].k < dqx)) break;", "if (!(o[t].k < 0.5 * dqx)) break;"),
    "search_scan_not_strict": ("if (!(o[t].k < dqx)) break;", "if (!(o[t].k <= dqx)) break;"),
    "beta_closed": ("if (in1 < t && in2 < t) blocked = 1;", "if (in1 <= t && in2 <= t) blocked = 1;"),
    "beta_one_ball": ("if (in1 < t && in2 < t) blocked = 1;", "if (in1 < t) blocked = 1;"),
    "beta_swapped_weights": ("double in1 = mu * a + lam * b;", "double in1 = lam * a + mu * b;"),
    "beta_radius_not_scaled": ("double t = lam * v;", "double t = v;"),
    "insert_pivot_no_removal": ("{ keep = 0; ++removed; }", "{ ++removed; }"),
    "insert_pivot_prune_too_far": ("double bi = mu[i] - 2.0 * ri, bj = mu[j] - 2.0 * rj;",
                                   "double bi = mu[i] - 3.0 * ri - 0.3 * mu[i], bj = mu[j] - 3.0 * rj - 0.3 * mu[j];"),
    "emst_wrong_endpoint": ("edges[2 * (e - 1)] = (int32_t)from[u];",
                            "edges[2 * (e - 1)] = (int32_t)(u > 0 ? u - 1 : 1);"),
}

RUNNER = r"""
import sys
sys.path.insert(0, {root!r})
import oracle
oracle.use_library({lib!r})
from tests import oracle_pins
failed = []
for chk in oracle_pins.ALL:
    try:
        chk(oracle)
    except AssertionError:
        failed.append(chk.__name__)
print("FAILED:" + ",".join(failed))
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "m.c")
        lib = os.path.join(td, "libm.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                        "-o", lib, c, "-lm"], check=True)
        out = subprocess.run([sys.executable, "-c", RUNNER.format(root=ROOT, lib=lib)],
                             capture_output=True, text=True, timeout=600)
        line = [l for l in out.stdout.splitlines() if l.startswith("FAILED:")]
        assert line, out.stdout + out.stderr
        assert line[0] != "FAILED:", f"no pin caught mutant {name}"
