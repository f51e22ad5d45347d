"""Seeded input generator: sizes, reproducibility, connectivity, load scaling."""
import numpy as np

from paper_2512_08465_gb300 import synth


def test_case118_sizes_and_classes():
    net = synth.case118()
    assert (net.n_bus, net.n_branch, net.n_gen) == (118, 186, 54)
    assert int((net.Pd_shape > 0).sum()) <= 99
    assert int((net.kind == synth.KIND_TRANSFORMER).sum()) == 11     # 175 lines + 11 transformers
    assert net.n_elem == 240
    assert net.ref_bus == int(net.gbus[0])


def test_seed_reproducible_and_distinct():
    a, b, c = synth.case118(), synth.case118(), synth.case118(seed=119)
    for k in ("f", "t", "r", "x", "b", "rate", "gbus", "Pmax", "Pd"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
    assert not np.array_equal(a.r, c.r)


def test_spanning_tree_connected_no_parallel():
    for seed in range(5):
        net = synth.make_network(40, 60, 10, 30, 2, seed=seed)
        parent = list(range(net.n_bus))

        def find(u):
            while parent[u] != u:
                u = parent[u]
            return u
        for a, b in zip(net.f, net.t):
            parent[find(int(a))] = find(int(b))
        assert len({find(u) for u in range(net.n_bus)}) == 1
        keys = {(min(a, b), max(a, b)) for a, b in zip(net.f, net.t)}
        assert len(keys) == net.n_branch and all(a != b for a, b in keys)


def test_load_levels_scale_total():
    net = synth.case118()
    for k, lv in enumerate(net.levels):
        assert abs(net.Pd[k].sum() - lv * net.Pmax.sum()) < 1e-6 * net.Pmax.sum()
        np.testing.assert_allclose(net.Qd[k], 0.3 * net.Pd[k])


def test_distributions_in_range():
    net = synth.case118()
    assert np.all((net.r >= 0.001) & (net.r <= 0.05))
    ratio = net.x / net.r
    assert np.all((ratio >= 3) & (ratio <= 10))
    assert np.all((net.Pmax >= 50) & (net.Pmax <= 500))
    np.testing.assert_allclose(net.Qmax, 0.5 * net.Pmax)
    assert np.all((net.H >= 2) & (net.H <= 8)) and np.all((net.D >= 0) & (net.D <= 2))


def test_pairs_and_scenario_count_identity():
    # Section I / V: 239 elements give 1 + 239 + 239*238 = 57,122 ordered scenarios.
    E = 239
    i, j = synth.all_pairs(E)
    assert len(i) == E * (E - 1) // 2
    assert 1 + E + 2 * len(i) == 57122
    assert np.all(i < j)
