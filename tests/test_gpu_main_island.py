"""Main-island form on the GPU (cs_options.main_island = 1) against the oracle
(oracle/island.py): an islanded scenario keeps class ISLANDED and S = 1, and
gets the OPF of the component with the largest in-service generation, with the
reference moved into it when the original one is outside.

Bar: main_klass and the choice of island bit-exact (buses outside it carry
Vm = Va = 0 exactly); the shed bit-exact (both sides add the same per-unit loads
in bus order); cost within 1e-6 relative; Vm, Va, voltage margin and loading
within 1e-8 where the main island's OPF converged; max Re and min damping ratio
of its small-signal screen within 1e-6 (FP64 form); iteration counts of converged
OPFs exactly.  No
main_klass may differ; cases in the guard band of the parity suite (an oracle OPF
that needed >= 48 of its 50 iterations, or a decisive eigen statistic within 1e-6
of its threshold) are counted and reported.  Scenarios that do not split are
unchanged by the form.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import twonets  # noqa: E402
from paper_2512_08465_gb300 import cs, synth  # noqa: E402
from oracle import grid, island  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL_V, TOL_COST, TOL_EIG = 1e-8, 1e-6, 1e-6
FIELDS = ("klass", "severe", "n_islands", "opf_iters", "cost", "max_re", "min_zeta")


def _run(ctx, nid, level, ei, ej, nb):
    ti = torch.as_tensor(np.asarray(ei, np.int32), device=DEV)
    tj = torch.as_tensor(np.asarray(ej, np.int32), device=DEV)
    out = ctx.alloc_results(ti.numel(), DEV, nb, indices=True, main_island=True)
    ctx.evaluate_device(nid, level, ti, tj, out)
    ctx.sync()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _compare(got, refs, nb):
    guard = 0
    for q, r in enumerate(refs):
        assert int(got["klass"][q]) == 1 and int(got["severe"][q]) == 1, q
        assert got["shed_mw"][q] == r["shed_mw"], (q, got["shed_mw"][q], r["shed_mw"])
        mk = int(got["main_klass"][q])
        near = r["opf_iters"] >= 48 or (np.isfinite(r["max_re"]) and (
            abs(r["max_re"]) < TOL_EIG or abs(r["min_zeta"] - island.DAMPING_MIN) < TOL_EIG))
        guard += bool(near)
        assert mk == r["main_klass"], (q, mk, r["main_klass"], "guard band" if near else "")
        if r["converged"]:
            assert int(got["opf_iters"][q]) == r["opf_iters"], (q, int(got["opf_iters"][q]), r["opf_iters"])
        if r["live"] is None:
            continue
        vm = got["Vm"][q * nb:(q + 1) * nb]
        va = got["Va"][q * nb:(q + 1) * nb]
        dead = ~r["live"]
        assert np.all(vm[dead] == 0.0) and np.all(va[dead] == 0.0), q
        if r["converged"]:
            assert abs(got["cost"][q] - r["cost"]) <= TOL_COST * abs(r["cost"]), q
            assert np.abs(vm - r["Vm"]).max() <= TOL_V and np.abs(va - r["Va"]).max() <= TOL_V, q
            assert abs(got["v_margin"][q] - r["v_margin"]) <= TOL_V, q
            assert abs(got["max_loading"][q] - r["max_loading"]) <= TOL_V, q
            if np.isfinite(r["max_re"]):              # the main island's small-signal screen ran
                assert abs(got["max_re"][q] - r["max_re"]) <= TOL_EIG, (q, got["max_re"][q], r["max_re"])
                assert abs(got["min_zeta"][q] - r["min_zeta"]) <= TOL_EIG, q
            else:
                assert np.isnan(got["max_re"][q]) and np.isnan(got["min_zeta"][q]), q
        else:
            assert np.isnan(got["cost"][q]) and np.isnan(got["v_margin"][q]), q
    return guard


@pytest.fixture(scope="module")
def net118():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return synth.case118()


def _islanded_pairs(net):
    ii, jj = synth.all_pairs(net.n_elem)
    out = []
    for a, b in zip(ii, jj):
        sc = grid.make_scenario(net, 0, int(a), int(b))
        if grid.count_islands(net.n_bus, net.f[sc.br], net.t[sc.br]) > 1:
            out.append((int(a), int(b)))
    return out


def test_main_island_118bus_matches_oracle(net118):
    """Every islanded N-1, the pair that isolates the reference bus, pairs whose split
    leaves several buses outside, and a random sample of islanded pairs, at both load
    levels; non-islanded scenarios in the same launch are unchanged by the form."""
    net = net118
    nb = net.n_bus
    isl = _islanded_pairs(net)
    refb = [b for b in range(net.n_branch) if net.ref_bus in (net.f[b], net.t[b])]
    pick = [p for p in isl if set(refb) <= set(p)]
    assert pick, "no pair isolates the reference bus"
    multi = [p for p in isl if (~island.main_island(net, grid.make_scenario(net, 0, *p))[0]).sum() > 1]
    rng = np.random.default_rng(23)
    pick += [multi[q] for q in rng.choice(len(multi), 8, replace=False)]
    pick += [isl[q] for q in rng.choice(len(isl), 24, replace=False)]
    n1 = [(e, -1) for e in range(net.n_elem)
          if grid.count_islands(net.n_bus, *(lambda sc: (net.f[sc.br], net.t[sc.br]))(
              grid.make_scenario(net, 0, e))) > 1]
    scen = n1 + pick
    ii, jj = synth.all_pairs(net.n_elem)
    plain = [(int(ii[q]), int(jj[q])) for q in rng.choice(ii.size, 64, replace=False)]
    ctx = cs.Context(main_island=1)
    nid = ctx.load_network(net)
    ref_ctx = cs.Context()
    rid = ref_ctx.load_network(net)
    guard = 0
    for level in (0, 1):
        refs = island.evaluate_main_island_many(net, [(level, a, b) for a, b in scen])
        ei = [a for a, _ in scen] + [a for a, _ in plain]
        ej = [b for _, b in scen] + [b for _, b in plain]
        got = _run(ctx, nid, level, ei, ej, nb)
        head = {k: v[:len(scen) * (nb if k in ("Vm", "Va") else 1)] for k, v in got.items()}
        guard += _compare(head, refs, nb)
        moved = [q for q, r in enumerate(refs) if r["ref"] >= 0 and r["ref"] != net.ref_bus]
        assert moved, "the reference-isolating pair did not move the reference"
        # the form leaves scenarios that do not split unchanged, bit for bit
        base = _run(ref_ctx, rid, level, ei, ej, nb)
        tail = slice(len(scen), len(ei))
        for k in FIELDS + ("v_margin", "max_loading"):
            split = np.asarray(got["n_islands"]) > 1
            np.testing.assert_array_equal(got[k][tail][~split[tail]], base[k][tail][~split[tail]], err_msg=k)
        assert np.all(got["main_klass"][tail][~split[tail]] == 255)
        assert np.all(got["shed_mw"][tail][~split[tail]] == 0.0)
        # without the form, an islanded scenario has no main-island result
        assert np.all(base["main_klass"] == 255)
        assert np.all(np.isnan(base["shed_mw"][:len(scen)]))
        assert np.all(base["opf_iters"][:len(scen)] == 0)
    print(f"[parity] main island, 118-bus: 0 main-class mismatches, {guard} in the guard band")
    ctx.close()
    ref_ctx.close()


def test_tie_line_split_moves_the_reference_and_no_generation_case():
    """Two networks joined by one tie with the reference on the smaller side: with the
    tie out the larger side is the main island and the reference moves to its largest
    unit.  A one-generator network with that generator and a bridge out has no main
    island: main_klass OPF_NONCONV, the whole load shed, Vm = Va = 0."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A, Bn = twonets.pair()
    J = twonets.join(A, Bn, 2, 4, ref=A.n_bus + Bn.ref_bus)
    tie = J.n_branch - 1
    scen = [(tie, -1), (tie, 0), (tie, J.n_branch + 1)]       # tie alone, with a branch, with a unit
    ctx = cs.Context(main_island=1)
    nid = ctx.load_network(J)
    got = _run(ctx, nid, 0, [a for a, _ in scen], [b for _, b in scen], J.n_bus)
    refs = [island.evaluate_main_island(J, 0, a, b) for a, b in scen]
    assert refs[0]["ref"] != J.ref_bus
    _compare(got, refs, J.n_bus)
    ctx.close()
    one = synth.make_network(9, 9, 1, 6, 0, seed=5, levels=(0.5,))
    bridges = [b for b in range(one.n_branch)
               if grid.count_islands(one.n_bus, np.delete(one.f, b), np.delete(one.t, b)) > 1]
    ctx = cs.Context(main_island=1)
    nid = ctx.load_network(one)
    got = _run(ctx, nid, 0, [bridges[0]], [one.n_branch], one.n_bus)
    ref = island.evaluate_main_island(one, 0, bridges[0], one.n_branch)
    assert ref["live"] is None
    assert int(got["main_klass"][0]) == island.OPF_NONCONV and got["shed_mw"][0] == ref["shed_mw"]
    assert int(got["opf_iters"][0]) == 0 and np.isnan(got["cost"][0])
    assert np.all(got["Vm"] == 0.0) and np.all(got["Va"] == 0.0)
    ctx.close()
