"""Pins of the main-island oracle (oracle/island.py).

Two networks are built apart and joined here by one tie branch, by a
construction of this test's own.  With the tie out, the main island is the
network with the larger generation: its OPF must be that network's standalone
OPF, and the shed must be the other network's load.  The reference is
re-assigned when it falls outside the main island; the angles then move by one
constant and nothing else changes.
"""
import copy

import numpy as np

import twonets
from paper_2512_08465_gb300 import synth
from oracle import grid, island, opf, pipeline


def _standalone(net):
    return opf.solve(net, grid.make_scenario(net, 0))


def _check_equal_opf(r, ref_net, live_slice, same_ref):
    s = _standalone(ref_net)
    assert s["converged"] and r["converged"]
    assert abs(r["cost"] - s["cost"]) <= 1e-6 * abs(s["cost"])
    np.testing.assert_allclose(r["Vm"][live_slice], s["Vm"], atol=1e-6)
    d = r["Va"][live_slice] - s["Va"]
    if same_ref:
        np.testing.assert_allclose(d, 0.0, atol=1e-6)
    else:
        assert np.ptp(d) < 1e-6                      # one constant: the reference moved
    # the small-signal screen of the main island is the standalone network's (a common
    # angle shift moves no eigenvalue)
    p = pipeline.evaluate(ref_net, 0)
    assert r["main_klass"] == p["klass"]
    if np.isfinite(p["max_re"]):
        assert abs(r["max_re"] - p["max_re"]) <= 1e-6 and abs(r["min_zeta"] - p["min_zeta"]) <= 1e-6


def test_labels_are_components_in_lowest_bus_order():
    for seed in range(5):
        net = synth.make_network(20, 22, 4, 10, 0, seed=seed)
        rng = np.random.default_rng(seed)
        keep = rng.random(net.n_branch) > 0.25
        f, t = net.f[keep], net.t[keep]
        lab = island.island_labels(net.n_bus, f, t)
        assert np.all(lab[f] == lab[t])
        assert lab.max() + 1 == grid.count_islands(net.n_bus, f, t)
        first = [int(np.flatnonzero(lab == c)[0]) for c in range(lab.max() + 1)]
        assert first == sorted(first)


def test_tie_out_larger_generation_is_main_and_slack_moves():
    A, Bn = twonets.pair()
    assert A.Pmax.sum() > Bn.Pmax.sum()
    J = twonets.join(A, Bn, 2, 4, ref=A.n_bus + Bn.ref_bus)          # reference inside B
    tie = J.n_branch - 1
    r = island.evaluate_main_island(J, 0, tie)
    nA = A.n_bus
    assert r["live"][:nA].all() and not r["live"][nA:].any()
    assert r["ref"] == int(A.gbus[np.argmax(A.Pmax)])          # largest unit of the main island
    assert abs(r["Va"][r["ref"]]) < 1e-12 and np.all(r["Vm"][nA:] == 0.0)
    assert abs(r["shed_mw"] - Bn.Pd[0].sum()) <= 1e-9 * Bn.Pd[0].sum()
    _check_equal_opf(r, A, slice(0, nA), same_ref=False)
    assert np.isfinite(r["max_re"])                           # the screen ran on the main island


def test_reference_kept_when_inside_main_island():
    A, Bn = twonets.pair()
    J = twonets.join(A, Bn, 2, 4, ref=A.ref_bus)
    r = island.evaluate_main_island(J, 0, J.n_branch - 1)
    assert r["ref"] == A.ref_bus
    _check_equal_opf(r, A, slice(0, A.n_bus), same_ref=True)


def test_swapping_generation_swaps_the_main_island():
    A, Bn = twonets.pair()
    Bn = copy.copy(Bn)
    for k in ("Pmax", "Qmax", "Qmin"):
        setattr(Bn, k, 10.0 * getattr(Bn, k))
    assert Bn.Pmax.sum() > A.Pmax.sum()
    J = twonets.join(A, Bn, 2, 4, ref=A.ref_bus)
    r = island.evaluate_main_island(J, 0, J.n_branch - 1)
    nA = A.n_bus
    assert r["live"][nA:].all() and not r["live"][:nA].any()
    assert r["ref"] == nA + int(Bn.gbus[np.argmax(Bn.Pmax)])
    assert abs(r["shed_mw"] - A.Pd[0].sum()) <= 1e-9 * A.Pd[0].sum()
    _check_equal_opf(r, Bn, slice(nA, J.n_bus), same_ref=False)


def test_equal_generation_picks_the_island_of_bus_zero():
    A, _ = twonets.pair()
    J = twonets.join(A, A, 1, 1, ref=A.n_bus + A.ref_bus)
    r = island.evaluate_main_island(J, 0, J.n_branch - 1)
    assert r["live"][:A.n_bus].all() and not r["live"][A.n_bus:].any()


def test_connected_scenario_is_not_islanded():
    A, _ = twonets.pair()
    r = island.evaluate_main_island(A, 0)
    assert r["main_klass"] == island.NOT_ISLANDED and r["shed_mw"] == 0.0 and r["opf_iters"] == 0


def test_no_generation_anywhere_means_no_main_island():
    net = synth.make_network(9, 9, 1, 6, 0, seed=5, levels=(0.5,))
    bridges = [b for b in range(net.n_branch)
               if grid.count_islands(net.n_bus, np.delete(net.f, b), np.delete(net.t, b)) > 1]
    assert bridges
    r = island.evaluate_main_island(net, 0, bridges[0], net.n_branch)    # the only generator out too
    assert r["live"] is None and r["main_klass"] == island.OPF_NONCONV
    assert abs(r["shed_mw"] - net.Pd[0].sum()) <= 1e-9 * net.Pd[0].sum()


def test_generator_outage_moves_the_main_island():
    """Same split, different generation: with the tie and A's largest unit out, B (now the
    larger total Pmax) is the main island although A has more buses."""
    A, Bn = twonets.pair()
    Bn = copy.copy(Bn)
    kA = int(np.argmax(A.Pmax))
    gap = A.Pmax.sum() - A.Pmax[kA]                       # A's capacity without its largest unit
    scale = 1.0 + (gap - Bn.Pmax.sum()) / Bn.Pmax.sum() + 0.2
    for k in ("Pmax", "Qmax", "Qmin"):
        setattr(Bn, k, scale * getattr(Bn, k))
    assert A.Pmax.sum() > Bn.Pmax.sum() > gap and A.n_bus > Bn.n_bus
    J = twonets.join(A, Bn, 2, 4, ref=A.ref_bus)
    tie = J.n_branch - 1
    assert island.evaluate_main_island(J, 0, tie)["live"][:A.n_bus].all()
    r = island.evaluate_main_island(J, 0, tie, J.n_branch + kA)
    assert r["live"][A.n_bus:].all() and not r["live"][:A.n_bus].any()
    assert r["ref"] == A.n_bus + int(Bn.gbus[np.argmax(Bn.Pmax)])
    assert abs(r["shed_mw"] - A.Pd[0].sum()) <= 1e-9 * A.Pd[0].sum()


def test_three_way_split_picks_the_largest_generation():
    """A - B - C chained by two ties; both ties out gives three islands, and the main one
    is the island with the largest total Pmax wherever it sits in the bus order."""
    A, Bn = twonets.pair()
    C = synth.make_network(9, 12, 3, 6, 0, seed=11, levels=(0.5,))
    C = copy.copy(C)
    for k in ("Pmax", "Qmax", "Qmin"):
        setattr(C, k, 3.0 * getattr(C, k))
    AB = twonets.join(A, Bn, 2, 4, ref=A.ref_bus)
    J = twonets.join(AB, C, A.n_bus + 1, 3, ref=A.ref_bus)   # second tie: a bus of B to a bus of C
    caps = [A.Pmax.sum(), Bn.Pmax.sum(), C.Pmax.sum()]
    assert int(np.argmax(caps)) == 2
    t1, t2 = AB.n_branch - 1, J.n_branch - 1
    r = island.evaluate_main_island(J, 0, t1, t2)
    assert grid.count_islands(J.n_bus, np.delete(J.f, [t1, t2]), np.delete(J.t, [t1, t2])) == 3
    nAB = AB.n_bus
    assert r["live"][nAB:].all() and not r["live"][:nAB].any()
    assert abs(r["shed_mw"] - (A.Pd[0].sum() + Bn.Pd[0].sum())) <= 1e-9 * (A.Pd[0].sum() + Bn.Pd[0].sum())
