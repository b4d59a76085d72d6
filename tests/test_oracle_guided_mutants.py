"""The checks of the guided oracle (the staged search and the membership-rule counts) must
catch plausible mistakes planted in a copy of oracle/guided_oracle.c.

Each mutant is a textual edit compiled with the unchanged definitions' file into a temporary
library; the checks of tests/test_oracle_guided.py run against it in a fresh process and at
least one must fail.  The committed oracle is never modified.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GUIDED = os.path.join(ROOT, "oracle", "guided_oracle.c")
DEFS = os.path.join(ROOT, "oracle", "grng_oracle.c")

MUTANTS = {
    # Stage II: the pivot's radius left out of both conditions (the domain taken as a point)
    "stage2_without_radii": ("const double a1 = dq[j] - F.radius[j], a2 = dq[j] - 2.0 * F.radius[j];",
                             "const double a1 = dq[j], a2 = dq[j];"),
    # Stage III: the distance of p_k to x bounded without x's distance to its pivot
    "stage3_bound_without_member": ("const double e2 = Dpp[(int64_t)k * m + j] + F.mdist[x];",
                                    "const double e2 = Dpp[(int64_t)k * m + j];"),
    # Stage VI: the visit stops at the first pivot farther than x, ignoring the domains' reach
    "stage6_stops_early": ("if (dqp - dmax_all >= dqx + G_MARGIN * (dqp + dmax_all + dqx)) break;\n"
                           "                        const int64_t pid = piv[p];",
                           "if (dqp >= dqx) break;\n"
                           "                        const int64_t pid = piv[p];"),
    # Stage I: a pivot kept when it is linked to any parent instead of every parent
    "stage1_any_parent": ("if (i != j && !F.gg[(int64_t)(i < j ? i : j) * m + (i < j ? j : i)]) ok = 0;",
                          "if (i != j && F.gg[(int64_t)(i < j ? i : j) * m + (i < j ? j : i)]) { ok = 1; break; } "
                          "else ok = 0;"),
    # membership rule B: a pair kept when one parent pair is linked instead of all of them
    "rule_b_one_parent_pair": ("if (p != q && !B.gg[(int64_t)(p < q ? p : q) * mb + (p < q ? q : p)]) in_b = 0;",
                               "if (p == q || B.gg[(int64_t)(p < q ? p : q) * mb + (p < q ? q : p)]) in_b = 1; "
                               "else if (s == 0 && t == 0) in_b = 0;"),
}

RUNNER = r"""
import sys
sys.path.insert(0, {root!r})
import oracle
oracle.use_library({lib!r})
from tests import test_oracle_guided as T
failed = []
for name in ("test_search_by_stages_equals_definition", "test_search_by_stages_on_the_workload_generators",
             "test_candidate_rules_sound_and_restated"):
    try:
        getattr(T, name)()
    except AssertionError:
        failed.append(name)
print("FAILED:" + ",".join(failed))
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_guided_checks_catch_mutant(name):
    old, new = MUTANTS[name]
    src = open(GUIDED).read()
    assert src.count(old) == 1, f"mutation site for {name} not found"
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "g.c")
        lib = os.path.join(td, "libg.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                        "-o", lib, DEFS, c, "-lm"], check=True)
        out = subprocess.run([sys.executable, "-c", RUNNER.format(root=ROOT, lib=lib)],
                             capture_output=True, text=True, timeout=600)
        line = [l for l in out.stdout.splitlines() if l.startswith("FAILED:")]
        assert line, out.stdout + out.stderr
        assert line[0] != "FAILED:", f"no check caught mutant {name}"
