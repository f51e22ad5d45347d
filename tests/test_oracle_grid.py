"""Oracle islanding and admittance matrices against independent routes."""
import itertools

import numpy as np
import pytest

from paper_2512_08465_gb300 import synth
from oracle import grid


def _components_union(n, edges):
    parent = list(range(n))

    def find(u):
        while parent[u] != u:
            parent[u] = parent[parent[u]]
            u = parent[u]
        return u
    for a, b in edges:
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[ra] = rb
    return len({find(u) for u in range(n)})


def test_islands_bruteforce_all_edge_subsets():
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = int(rng.integers(2, 7))
        allp = [(a, b) for a in range(n) for b in range(a + 1, n)]
        m = int(rng.integers(1, len(allp) + 1))
        idx = rng.choice(len(allp), m, replace=False)
        edges = [allp[k] for k in idx]
        for r in range(len(edges) + 1):
            for keep in itertools.combinations(range(len(edges)), r):
                e = [edges[k] for k in keep]
                f = [a for a, _ in e]
                t = [b for _, b in e]
                assert grid.count_islands(n, f, t) == _components_union(n, e)


def test_isolated_bus_counts_as_island():
    assert grid.count_islands(3, [0], [1]) == 2
    assert grid.count_islands(1, [], []) == 1


def test_n1_islanding_iff_bridge():
    """An N-1 branch outage splits the network iff the branch is a bridge; bridges are
    found here by exhaustive deletion plus a reachability test of the two ends."""
    net = synth.case118()
    for k in range(net.n_branch):
        sc = grid.make_scenario(net, 0, k)
        nis = grid.count_islands(net.n_bus, net.f[sc.br], net.t[sc.br])
        # reachability of t from f without branch k, by plain DFS
        adj = {u: [] for u in range(net.n_bus)}
        for e in sc.br:
            adj[int(net.f[e])].append(int(net.t[e]))
            adj[int(net.t[e])].append(int(net.f[e]))
        src, dst = int(net.f[k]), int(net.t[k])
        seen, stack = {src}, [src]
        while stack:
            u = stack.pop()
            for w in adj[u]:
                if w not in seen:
                    seen.add(w)
                    stack.append(w)
        assert (nis > 1) == (dst not in seen)
        assert nis in (1, 2)


def test_generator_outage_keeps_topology():
    net = synth.case118()
    sc = grid.make_scenario(net, 0, net.n_branch + 3, net.n_branch + 7)
    assert len(sc.br) == net.n_branch and len(sc.gen) == net.n_gen - 2
    assert grid.count_islands(net.n_bus, net.f[sc.br], net.t[sc.br]) == 1


def test_ybus_row_sums_are_shunts():
    """With unit taps, Y 1 = bus shunts + half the line charging of incident branches."""
    net = synth.make_network(12, 18, 3, 8, 2, seed=4)
    net.Bs[:] = np.linspace(0, 5, net.n_bus)
    Y, Yf, Yt, Cf, Ct = grid.ybus(net, np.arange(net.n_branch))
    expect = 1j * net.Bs / net.base_mva
    for e in range(net.n_branch):
        expect[net.f[e]] += 0.5j * net.b[e]
        expect[net.t[e]] += 0.5j * net.b[e]
    np.testing.assert_allclose(Y.sum(axis=1), expect, atol=1e-12)
    np.testing.assert_allclose(Y, Y.T, atol=0)


def test_tap_branch_two_port():
    """Ideal transformer of ratio a on the from side in series with z: I_f = (V_f/a - V_t)/(z a)."""
    net = synth.make_network(2, 1, 1, 1, 0, seed=1)
    net.tap[:] = 1.05
    net.b[:] = 0.0
    yff, yft, ytf, ytt = grid.branch_admittances(net, np.array([0]))
    z = net.r[0] + 1j * net.x[0]
    Vf, Vt = 1.02 * np.exp(0.1j), 0.97 * np.exp(-0.05j)
    a = 1.05
    If = (Vf / a - Vt) / z / a
    It = (Vt - Vf / a) / z
    assert abs(yff[0] * Vf + yft[0] * Vt - If) < 1e-12
    assert abs(ytf[0] * Vf + ytt[0] * Vt - It) < 1e-12
