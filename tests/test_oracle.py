"""The FP64 oracle against its pins (CPU only)."""
import numpy as np
import pytest

import oracle
from . import oracle_pins


@pytest.mark.parametrize("check", oracle_pins.ALL, ids=lambda f: f.__name__)
def test_oracle_pin(check):
    check(oracle)


def test_degree_arithmetic():
    oracle_pins.degree_arithmetic()


def test_key_is_sequential_fp64_without_fma():
    # a case where a fused multiply-add or a different summation order changes the
    # last bit: the canonical value is the plain left-to-right double sum
    a = np.array([1e8, 1.0, -1e8, 3.0], np.float32)
    b = np.array([0.0, 0.0, 0.0, 0.0], np.float32)
    acc = 0.0
    for x in a.tolist():
        acc = acc + x * x
    assert oracle.key(a, b, oracle.L2) == acc
    assert oracle.key(a, b, oracle.L1) == ((1e8 + 1.0) + 1e8) + 3.0


def test_fixtures_agree_with_exact_checker():
    # the hand-derived fixtures and the exact rational checker are two independent
    # readings of the same definitions
    import json
    from . import exact
    g = json.load(open(oracle_pins.GOLDEN))
    for ex in g["rng"]:
        assert set(map(tuple, ex["edges"])) == set(exact.rng(ex["points"], ex["metric"])), ex["name"]
    for ex in g["grng"]:
        assert set(map(tuple, ex["edges"])) == set(exact.grng(ex["points"], ex["radii"], ex["metric"])), ex["name"]
