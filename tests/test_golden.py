"""Stored values: the paper's printed constants, and the oracle's own results
on the tiny case (written by tests/golden/make_c0_golden.py, which calls only
oracle/ and workloads/)."""
import json
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def test_paper_constants_consistent_with_each_other():
    c = load("paper_constants.json")
    # Sec. IV quotes the accuracy limit both in micro-hartree and in meV; the
    # Sec. III conversion factor must map one onto the other
    mev = c["accuracy_limit_uEh"]["value"] * 1e-6 * c["hartree_eV"]["value"] * 1e3
    assert round(mev, 2) == c["accuracy_limit_meV"]["value"]


def test_code_uses_the_paper_constants():
    import bench
    from oracle import qp

    c = load("paper_constants.json")
    assert bench.HARTREE_EV == c["hartree_eV"]["value"]
    # the Newton threshold the oracle and the benchmark default to is Eq. NR's
    assert qp.newton_qp.__defaults__[0] == c["newton_delta_Ha"]["value"]


@pytest.fixture(scope="module")
def golden_c0():
    return load("c0_oracle.json")


def test_oracle_reproduces_stored_c0(golden_c0):
    """Regression pin: a change to the oracle's arithmetic shows up here."""
    import sys
    sys.path.insert(0, HERE)
    import make_c0_golden

    now = make_c0_golden.compute()
    g = golden_c0
    assert now["cd"]["M"] == g["cd"]["M"]
    assert now["cd"]["piv"] == g["cd"]["piv"]
    np.testing.assert_allclose(now["sigma_at_eps"], g["sigma_at_eps"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(now["dsigma_at_eps"], g["dsigma_at_eps"], rtol=1e-12)
    for a, b in zip(now["qp"], g["qp"]):
        assert a["iters"] == b["iters"] and a["status"] == b["status"]
        assert a["omega"] == pytest.approx(b["omega"], abs=1e-12)
        assert a["pole"] == pytest.approx(b["pole"], rel=1e-10)


def test_stored_c0_invariants(golden_c0):
    """The stored decomposition and poles satisfy what the method fixes."""
    g = golden_c0
    assert len(set(g["cd"]["piv"])) == g["cd"]["M"]               # distinct pivots
    assert g["cd"]["max_residual"] <= g["delta"]                   # stop rule
    assert all(s < 0 for s in g["dsigma_at_eps"])                  # Sigma' < 0
    for r in g["qp"]:
        assert r["status"] == 0 and 0 < r["pole"] <= 1             # 0 < P <= 1
