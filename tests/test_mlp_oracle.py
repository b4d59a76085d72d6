"""CPU checks of the FP64 interceptor-ranking network (oracle/mlp_oracle.c): its pins,
and that the pins catch mistakes planted in a copy of it."""
import os
import subprocess
import sys
import tempfile

import pytest

import oracle
from tests import mlp_pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mlp_oracle.c")


@pytest.mark.parametrize("pin", mlp_pins.ALL, ids=lambda f: f.__name__)
def test_mlp_pin(pin):
    pin(oracle)


MUTANTS = {
    "relu_leaks": ("h1[j] = a > 0.0 ? a : 0.0;", "h1[j] = a > 0.0 ? a : 0.01 * a;"),
    "layer1_kink_dropped": ("d1[i] = z1[i] > 0.0 ? a : 0.0;", "d1[i] = a;"),
    "w2_transposed_in_backprop": ("a += P[OFF_W2 + j * MLP_H + i] * d2[j];", "a += P[OFF_W2 + i * MLP_H + j] * d2[j];"),
    "loss_sign": ("const double ds = wb * (1.0 / (1.0 + exp(-s)) - y[b]) / (double)N;",
                  "const double ds = wb * (y[b] - 1.0 / (1.0 + exp(-s))) / (double)N;"),
    "bias2_dropped": ("double a = P[OFF_B2 + j];", "double a = 0.0;"),
    "weight_ignored_in_loss": ("loss += wb * (softplus(s) - y[b] * s);", "loss += softplus(s) - y[b] * s;"),
}

RUNNER = r"""
import sys
sys.path.insert(0, {root!r})
import oracle
oracle.use_library({lib!r})
from tests import mlp_pins
failed = []
for chk in mlp_pins.ALL:
    try:
        chk(oracle)
    except AssertionError:
        failed.append(chk.__name__)
print("FAILED:" + ",".join(failed))
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mlp_pins_catch_mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found"
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "m.c")
        lib = os.path.join(td, "libm.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                        "-o", lib, c, os.path.join(ROOT, "oracle", "grng_oracle.c"), "-fopenmp", "-lm"],
                       check=True)
        out = subprocess.run([sys.executable, "-c", RUNNER.format(root=ROOT, lib=lib)],
                             capture_output=True, text=True, timeout=300)
        line = [l for l in out.stdout.splitlines() if l.startswith("FAILED:")]
        assert line, out.stdout + out.stderr
        assert line[0] != "FAILED:", f"no pin caught mutant {name}"
