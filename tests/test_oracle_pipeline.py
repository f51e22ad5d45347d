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


def test_n3_scenarios_reduce_to_n2_and_are_order_free():
    """N-3 extension of the enumeration: a triple with a repeated or absent third
    element is the pinned N-2 scenario, and the result does not depend on the order
    of the three elements."""
    from oracle import grid, pipeline
    from paper_2512_08465_gb300 import synth
    net = synth.make_network(9, 12, 3, 6, 0, seed=5, levels=(0.5,))
    a = pipeline.evaluate(net, 0, 1, 7)
    for k in (-1, 1, 7):
        b = pipeline.evaluate(net, 0, 1, 7, k=k)
        assert b["klass"] == a["klass"] and b["n_islands"] == a["n_islands"] and b["opf_iters"] == a["opf_iters"]
    sc = grid.make_scenario(net, 0, 2, 9, 13)
    assert sc.out_elems == (2, 9, 13) and 13 - net.n_branch not in sc.gen and 2 not in sc.br
    r0 = pipeline.evaluate(net, 0, 2, 9, k=13)
    for (i, j, k) in ((13, 2, 9), (9, 13, 2)):
        r = pipeline.evaluate(net, 0, i, j, k=k)
        assert r["klass"] == r0["klass"] and r["opf_iters"] == r0["opf_iters"]
        if r0["converged"]:
            assert r["cost"] == r0["cost"]


def test_classification_truth_table(monkeypatch):
    """Section II-B: a scenario is severe when at least one criterion fails, and the
    class is the first failing criterion in the order islanding, OPF convergence,
    operational limits, eigenvalue iteration, Re >= 0, damping below the threshold.
    Every combination of outcomes is forced by stubbing the criteria themselves."""
    import itertools
    from oracle import dynamics, eig, opf
    net = synth.make_network(9, 12, 3, 6, 0, seed=5, levels=(0.5,))
    order = ("island", "nonconv", "limit", "eigfail", "unstable", "damped")
    klass = {"island": pipeline.ISLANDED, "nonconv": pipeline.OPF_NONCONV, "limit": pipeline.LIMIT,
             "eigfail": pipeline.EIG_FAIL, "unstable": pipeline.SS_UNSTABLE, "damped": pipeline.SS_POORLY_DAMPED}
    nb = net.n_bus
    for bits in itertools.product((False, True), repeat=len(order)):
        fail = dict(zip(order, bits))
        monkeypatch.setattr(grid, "count_islands", lambda n, f, t, v=fail["island"]: 2 if v else 1)
        monkeypatch.setattr(opf, "solve", lambda net_, sc, v=fail["nonconv"]: dict(
            converged=not v, iterations=7, cost=1.0, Va=np.zeros(nb), Vm=np.ones(nb),
            Pg=np.zeros(3), Qg=np.zeros(3), conds=(0, 0, 0, 0)))
        monkeypatch.setattr(opf, "severity_indices", lambda r: (0.01, 0.5))
        monkeypatch.setattr(opf, "limit_violation", lambda r, v=fail["limit"]: v)

        class _M:
            def __init__(self, *a):
                pass

            def reduced_state_matrix(self):
                return np.zeros((2, 2))
        monkeypatch.setattr(dynamics, "Model", _M)
        re = 0.1 if fail["unstable"] else -0.5
        zeta = 0.01 if fail["damped"] else 0.3
        lam = np.array([complex(re, 1.0), complex(-zeta, np.sqrt(1 - zeta * zeta))])
        monkeypatch.setattr(eig, "eigvals", lambda A, v=fail["eigfail"], lam=lam: (lam, not v, 3))
        r = pipeline.evaluate(net, 0, 1, 2)
        first = next((k for k in order if fail[k]), None)
        want = pipeline.SECURE if first is None else klass[first]
        assert r["klass"] == want, (fail, r["klass"])
        assert r["severe"] == int(any(bits)), fail
