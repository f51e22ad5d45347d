"""Oracle scenario pipeline: base case security and class semantics."""
import numpy as np
import pytest

from paper_2512_08465_gb300 import synth
from oracle import grid, pipeline


@pytest.fixture(scope="module")
def net():
    return synth.case118()


@pytest.mark.parametrize("level", [0, 1])
def test_base_case_is_secure(net, level):
    """Section II-A step 1: the pre-contingency state must be secure."""
    r = pipeline.evaluate(net, level)
    assert r["klass"] == pipeline.SECURE and r["severe"] == 0
    assert r["max_re"] < 0 and r["min_zeta"] >= pipeline.DAMPING_MIN


def test_islanding_scenario_skips_opf(net):
    bridges = [k for k in range(net.n_branch)
               if grid.count_islands(net.n_bus, np.delete(net.f, k), np.delete(net.t, k)) > 1]
    assert bridges
    r = pipeline.evaluate(net, 0, bridges[0])
    assert r["klass"] == pipeline.ISLANDED and r["severe"] == 1 and r["opf_iters"] == 0
    assert r["n_islands"] == 2


def test_damping_threshold_zero_is_the_literal_rule(net):
    """With damping_min = 0 only a non-negative real part makes the screen fail."""
    r = pipeline.evaluate(net, 0, -1, -1, damping_min=0.0)
    assert r["klass"] == pipeline.SECURE
    r = pipeline.evaluate(net, 0, -1, -1, damping_min=0.5)
    assert r["klass"] == pipeline.SS_POORLY_DAMPED


def test_pair_order_irrelevant(net):
    a = pipeline.evaluate(net, 0, 3, net.n_branch + 2)
    b = pipeline.evaluate(net, 0, net.n_branch + 2, 3)
    assert a["klass"] == b["klass"] and a["cost"] == b["cost"]
