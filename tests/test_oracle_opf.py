"""Oracle AC-OPF: derivatives, closed forms and optimality conditions."""
import numpy as np
import pytest

from paper_2512_08465_gb300 import synth
from oracle import grid, opf


def _fd_check(prob, x, lam, mu, eps=1e-6):
    f, df, g, h, Jg, Jh, c = prob.evaluate(x)
    Jg_fd = np.zeros_like(Jg)
    Jh_fd = np.zeros_like(Jh)
    df_fd = np.zeros_like(df)
    H_fd = np.zeros((prob.nx, prob.nx))

    def Lx(xx):
        _, d, _, _, G, Hh, _ = prob.evaluate(xx)
        return d + G.T @ lam + Hh.T @ mu
    for k in range(prob.nx):
        xp, xm = x.copy(), x.copy()
        xp[k] += eps
        xm[k] -= eps
        fp, _, gp, hp, *_ = prob.evaluate(xp)
        fm, _, gm, hm, *_ = prob.evaluate(xm)
        Jg_fd[:, k] = (gp - gm) / (2 * eps)
        Jh_fd[:, k] = (hp - hm) / (2 * eps)
        df_fd[k] = (fp - fm) / (2 * eps)
        H_fd[:, k] = (Lx(xp) - Lx(xm)) / (2 * eps)
    H = prob.hessian(c, lam, mu)
    return (np.abs(Jg - Jg_fd).max(), np.abs(Jh - Jh_fd).max(),
            np.abs(df - df_fd).max() / np.abs(df).max(), np.abs(H - H_fd).max() / np.abs(H).max(),
            np.abs(H - H.T).max())


@pytest.mark.parametrize("tap", [1.0, 0.97])
def test_derivatives_match_central_differences(tap):
    net = synth.make_network(9, 12, 3, 6, 1, seed=5, levels=(0.5,))
    net.tap[::3] = tap
    net.Bs[2] = 30.0
    prob = opf.Problem(net, grid.make_scenario(net, 0))
    rng = np.random.default_rng(0)
    x = prob.x0()
    x[:prob.nb] = rng.normal(0, 0.1, prob.nb)
    x[prob.nb:2 * prob.nb] = rng.uniform(0.95, 1.05, prob.nb)
    x[2 * prob.nb:] = rng.uniform(0, 1, 2 * prob.ng)
    lam = rng.normal(size=prob.neq)
    mu = rng.uniform(size=prob.niq)
    eg, eh, ef, eH, asym = _fd_check(prob, x, lam, mu)
    assert eg < 1e-6 and eh < 1e-6 and ef < 1e-8 and eH < 1e-6
    assert asym < 1e-9


def _two_bus(r, x, load_mw, load_mvar, gens):
    net = synth.make_network(2, 1, len(gens), 1, 0, seed=7, levels=(0.5,))
    net.r[:] = r
    net.x[:] = x
    net.b[:] = 0.0
    net.rate[:] = 1e5
    net.Pd_shape[:] = [0.0, load_mw]
    net.Qd_shape[:] = [0.0, load_mvar]
    net.Pd = net.Pd_shape[None, :].copy()
    net.Qd = net.Qd_shape[None, :].copy()
    for k, (bus, pmax, c2, c1) in enumerate(gens):
        net.gbus[k] = bus
        net.Pmax[k] = pmax
        net.Qmax[k] = 0.5 * pmax
        net.Qmin[k] = -0.5 * pmax
        net.c2[k] = c2
        net.c1[k] = c1
    net.ref_bus = int(net.gbus[0])
    return net


def test_two_bus_power_flow_closed_form():
    """Load P + jQ fed over r + jx from bus 0: |V2|^4 + (2(rP + xQ) - |V1|^2)|V2|^2
    + (r^2 + x^2)(P^2 + Q^2) = 0 must hold at the OPF solution."""
    net = _two_bus(0.02, 0.08, 400.0, 150.0, [(0, 2000.0, 0.01, 20.0)])
    r = opf.solve(net, grid.make_scenario(net, 0))
    assert r["converged"]
    P, Q = 400.0 / net.base_mva, 150.0 / net.base_mva
    v1, v2 = r["Vm"][0], r["Vm"][1]
    res = v2 ** 4 + (2 * (0.02 * P + 0.08 * Q) - v1 ** 2) * v2 ** 2 + (0.02 ** 2 + 0.08 ** 2) * (P * P + Q * Q)
    assert abs(res) < 1e-8
    # generation = load + series loss |I|^2 r
    I2 = (P * P + Q * Q) / v2 ** 2
    assert abs(r["Pg"][0] - (P + I2 * 0.02)) < 1e-8
    # the cost pushes voltages up to cut losses: the sending end sits at its bound
    assert abs(v1 - 1.06) < 1e-6


def test_two_generator_lossless_dispatch_closed_form():
    """r = 0: generation equals load, and the optimum equalises marginal costs."""
    c2a, c1a, c2b, c1b = 0.02, 15.0, 0.01, 25.0
    PL = 500.0
    net = _two_bus(0.0, 0.05, PL, 50.0, [(0, 1000.0, c2a, c1a), (1, 1000.0, c2b, c1b)])
    r = opf.solve(net, grid.make_scenario(net, 0))
    assert r["converged"]
    lam = (PL + c1a / (2 * c2a) + c1b / (2 * c2b)) / (1 / (2 * c2a) + 1 / (2 * c2b))
    Pa = (lam - c1a) / (2 * c2a)
    Pb = (lam - c1b) / (2 * c2b)
    B = net.base_mva
    assert abs(r["Pg"][0] * B - Pa) < 1e-5 and abs(r["Pg"][1] * B - Pb) < 1e-5
    cost = c2a * Pa ** 2 + c1a * Pa + c2b * Pb ** 2 + c1b * Pb
    assert abs(r["cost"] - cost) / cost < 1e-8


def test_kkt_conditions_at_converged_points():
    """Stationarity with finite-difference Jacobians, primal feasibility and
    complementarity at converged 118-bus points (base and two N-1 cases)."""
    net = synth.case118()
    for (lv, i) in ((0, -1), (0, 5), (1, 100)):
        sc = grid.make_scenario(net, lv, i)
        r = opf.solve(net, sc)
        assert r["converged"]
        prob = r["prob"]
        x = np.concatenate([r["Va"], r["Vm"], r["Pg"], r["Qg"]])
        f, df, g, h, Jg, Jh, _ = prob.evaluate(x)
        eps = 1e-7
        Lx = df.copy()
        for k in range(prob.nx):
            xp, xm = x.copy(), x.copy()
            xp[k] += eps
            xm[k] -= eps
            _, _, gp, hp, *_ = prob.evaluate(xp)
            _, _, gm, hm, *_ = prob.evaluate(xm)
            Lx[k] += r["lam"] @ ((gp - gm) / (2 * eps)) + r["mu"] @ ((hp - hm) / (2 * eps))
        scale = 1 + max(np.abs(r["lam"]).max(), np.abs(r["mu"]).max())
        assert np.abs(Lx).max() / scale < 1e-6
        assert np.abs(g).max() < 1e-7 and h.max() < 1e-7
        assert np.all(r["z"] > 0) and np.all(r["mu"] > 0)
        assert float(r["z"] @ r["mu"]) / (1 + np.abs(x).max()) < 1e-8
        assert not opf.limit_violation(r)


def test_infeasible_scenario_does_not_converge():
    """Load beyond total capacity has no feasible point."""
    net = _two_bus(0.01, 0.05, 1500.0, 100.0, [(0, 1000.0, 0.01, 20.0)])
    r = opf.solve(net, grid.make_scenario(net, 0))
    assert not r["converged"]


def test_severity_indices_at_binding_limits():
    """Non-binary severity indices pinned by optimality: a cheap generator behind a
    line rated below the load must push that line to its limit (loading 1), and a
    lossy line feeding a load from one generator drives the generator bus to Vmax
    (losses fall with voltage), so the voltage margin is 0."""
    from oracle import grid
    # congestion: cheap generator at bus 0, expensive at bus 1, load 300 MW at bus 1, rating 200 MVA
    net = _two_bus(0.0, 0.05, 300.0, 0.0, [(0, 500.0, 0.01, 10.0), (1, 500.0, 0.01, 40.0)])
    net.rate[:] = 200.0
    r = opf.solve(net, grid.make_scenario(net, 0))
    assert r["converged"]
    margin, loading = opf.severity_indices(r)
    assert abs(loading - 1.0) <= 1e-6 and margin >= -1e-8
    # losses: one generator, lossy line, load at the far end; Vm0 goes to Vmax
    net = _two_bus(0.02, 0.06, 150.0, 30.0, [(0, 500.0, 0.01, 20.0)])
    r = opf.solve(net, grid.make_scenario(net, 0))
    assert r["converged"]
    margin, loading = opf.severity_indices(r)
    assert abs(r["Vm"][0] - net.Vmax[0]) <= 1e-6 and abs(margin) <= 1e-6 and loading < 1.0


def test_conditions_hand_computed():
    """The four MIPS stopping quantities (Wang et al. 2007, Section III; the reading
    of the OPF of Section II-B-1) on numbers worked by hand:
      feasibility  max(|g|_inf, max h) / (1 + max(|x|_inf, |z|_inf)) = max(0.3, 0.2) / 5 = 0.06
      gradient     |Lx|_inf / (1 + max(|lam|_inf, |mu|_inf))          = 1.4 / 7           = 0.2
      complement.  z.mu / (1 + |x|_inf)                               = (1 + 1) / 5       = 0.4
      cost change  |f - f_prev| / (1 + |f_prev|)                      = 2 / 9
    The second case has every h < 0 (feasibility from g alone) and a cost drop."""
    x = np.array([3.0, -4.0])
    z = np.array([0.5, 2.0])
    g = np.array([0.1, -0.3])
    h = np.array([-0.5, 0.2])
    lam = np.array([1.0, -6.0])
    mu = np.array([2.0, 0.5])
    Lx = np.array([0.7, -1.4])
    feas, grad, comp, cost = opf.conditions(None, x, z, lam, mu, 10.0, 8.0, g, h, Lx)
    assert feas == pytest.approx(0.06, abs=1e-15)
    assert grad == pytest.approx(0.2, abs=1e-15)
    assert comp == pytest.approx(0.4, abs=1e-15)
    assert cost == pytest.approx(2.0 / 9.0, abs=1e-15)
    # all h negative: the largest |g| decides; |z| larger than |x|; cost falls from -4 to -7
    x = np.array([0.5])
    z = np.array([9.0, 1.0])
    g = np.array([-0.02])
    h = np.array([-3.0, -1.0])
    lam = np.array([0.0])
    mu = np.array([0.25, 0.75])
    Lx = np.array([-2.0])
    feas, grad, comp, cost = opf.conditions(None, x, z, lam, mu, -7.0, -4.0, g, h, Lx)
    assert feas == pytest.approx(0.02 / 10.0, abs=1e-15)     # 1 + max(0.5, 9)
    assert grad == pytest.approx(2.0 / 1.75, abs=1e-15)      # 1 + max(0, 0.75)
    assert comp == pytest.approx(3.0 / 1.5, abs=1e-15)       # 9*0.25 + 1*0.75 = 3
    assert cost == pytest.approx(3.0 / 5.0, abs=1e-15)


def test_iteration_stops_at_first_point_meeting_all_four_conditions():
    """The iteration count is the first iterate at which every condition is below
    the tolerance: the trace's previous iterate still fails one of them."""
    net = synth.case118()
    r = opf.solve(net, grid.make_scenario(net, 0, 5), trace=True)
    assert r["converged"] and r["iterations"] == len(r["hist"])
    last = r["hist"][-1][4:]
    prev = r["hist"][-2][4:]
    assert all(c < opf.TOL for c in last)
    assert any(c >= opf.TOL for c in prev)


def _forced(res, **changes):
    """A converged result with some limits of its problem moved (the point is
    unchanged); h is re-evaluated for the moved limits."""
    import copy
    prob = copy.copy(res["prob"])
    for k, v in changes.items():
        setattr(prob, k, v)
    x = np.concatenate([res["Va"], res["Vm"], res["Pg"], res["Qg"]])
    out = dict(res)
    out["prob"] = prob
    out["h"] = prob.evaluate(x)[3]
    return out


def test_limit_violation_forced_by_cutting_limits_below_the_point():
    """Section II-B-1: a converged point beyond an operational limit by more than
    1e-6 p.u. is a violation.  The two-bus point's sending-end flow is computed
    here from the voltages alone, |S_f| = |V_0 conj((V_0 - V_1)/(r + jx))|; a rating
    cut 3e-6 p.u. below it is violated, 0.5e-6 below it is within tolerance, and the
    same holds for Vmax, Pmax and Qmin moved across the point."""
    r_, x_ = 0.02, 0.08
    net = _two_bus(r_, x_, 400.0, 150.0, [(0, 2000.0, 0.01, 20.0)])
    res = opf.solve(net, grid.make_scenario(net, 0))
    assert res["converged"] and not opf.limit_violation(res)
    V = res["Vm"] * np.exp(1j * res["Va"])
    Sf = abs(V[0] * np.conj((V[0] - V[1]) / complex(r_, x_)))
    St = abs(V[1] * np.conj((V[1] - V[0]) / complex(r_, x_)))
    assert Sf > St                                    # the sending end carries the losses
    assert not opf.limit_violation(_forced(res, Smax2=np.array([(Sf - 0.5e-6) ** 2])))
    assert opf.limit_violation(_forced(res, Smax2=np.array([(Sf - 3e-6) ** 2])))
    assert not opf.limit_violation(_forced(res, Smax2=np.array([(Sf * 10.0) ** 2])))
    vmax = res["prob"].Vmax.copy()
    vmax[1] = res["Vm"][1] - 3e-6
    assert opf.limit_violation(_forced(res, Vmax=vmax))
    vmax[1] = res["Vm"][1] - 0.5e-6
    assert not opf.limit_violation(_forced(res, Vmax=vmax))
    assert opf.limit_violation(_forced(res, Pmax=res["Pg"] - 3e-6))
    assert not opf.limit_violation(_forced(res, Pmax=res["Pg"] - 0.5e-6))
    assert opf.limit_violation(_forced(res, Qmin=res["Qg"] + 3e-6))
    assert opf.limit_violation(_forced(res, Vmin=res["Vm"] + 3e-6))
