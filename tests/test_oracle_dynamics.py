"""Oracle small-signal model: equilibrium, Jacobian, Kron reduction, rotation mode."""
import numpy as np
import pytest

from paper_2512_08465_gb300 import synth
from oracle import dynamics, grid, opf


@pytest.fixture(scope="module")
def base118():
    net = synth.case118()
    sc = grid.make_scenario(net, 0)
    r = opf.solve(net, sc)
    assert r["converged"]
    return net, sc, r, dynamics.Model(net, sc, r["Va"], r["Vm"], r["Pg"], r["Qg"])


def test_equilibrium_is_a_fixed_point(base118):
    _, _, _, M = base118
    f0 = M.f_value(M.x0)
    assert np.abs(f0).max() < 1e-9


def test_state_matrix_matches_richardson_differences(base118):
    _, _, _, M = base118
    A = M.state_matrix()
    rng = np.random.default_rng(1)
    cols = rng.choice(A.shape[0], 25, replace=False)
    for k in cols:
        def d(h):
            xp, xm = M.x0.copy(), M.x0.copy()
            xp[k] += h
            xm[k] -= h
            return (M.f_value(xp) - M.f_value(xm)) / (2 * h)
        h = 1e-4
        rich = (4 * d(h / 2) - d(h)) / 3
        assert np.abs(rich - A[:, k]).max() < 1e-7 * max(1.0, np.abs(A).max())


def test_common_rotation_is_a_null_vector(base118):
    _, _, _, M = base118
    A = M.state_matrix()
    v0 = np.zeros(A.shape[0])
    v0[0::5] = 1.0
    assert np.abs(A @ v0).max() < 1e-9 * np.abs(A).max()


def test_angle_reference_removes_exactly_the_zero_mode(base118):
    """eig(A') = eig(A) less one zero (numpy used as a test-only cross-check)."""
    _, _, _, M = base118
    A = M.state_matrix()
    Ar = M.reduced_state_matrix()
    assert Ar.shape == (A.shape[0] - 1,) * 2
    wa = np.linalg.eigvals(A)
    wa = np.delete(wa, np.argmin(np.abs(wa)))
    wr = np.linalg.eigvals(Ar)
    for z in wr:
        k = int(np.argmin(np.abs(wa - z)))
        assert abs(wa[k] - z) < 1e-8 * np.abs(A).max()
        wa = np.delete(wa, k)
    assert np.abs(wr).min() > 1e-3


def test_reduced_matrix_matches_differences(base118):
    """A' by central differences of the reduced equations (angles relative to machine 0)."""
    _, _, _, M = base118
    Ar = M.reduced_state_matrix()
    m = M.m
    def f_red(xr):
        x = np.concatenate([[M.x0[0]], xr])
        for k in range(1, m):
            x[5 * k] = M.x0[0] + xr[5 * k - 1]
        fv = M.f_value(x)
        out = fv[1:].copy()
        for k in range(1, m):
            out[5 * k - 1] = fv[5 * k] - fv[0]
        return out
    xr0 = M.x0[1:].copy()
    for k in range(1, m):
        xr0[5 * k - 1] = M.x0[5 * k] - M.x0[0]
    assert np.abs(f_red(xr0)).max() < 1e-9
    rng = np.random.default_rng(2)
    for c in rng.choice(Ar.shape[0], 20, replace=False):
        h = 1e-4
        def d(hh):
            xp, xm = xr0.copy(), xr0.copy()
            xp[c] += hh
            xm[c] -= hh
            return (f_red(xp) - f_red(xm)) / (2 * hh)
        rich = (4 * d(h / 2) - d(h)) / 3
        assert np.abs(rich - Ar[:, c]).max() < 1e-7 * max(1.0, np.abs(Ar).max())


def test_kron_reduction_equals_full_nodal_solve(base118):
    """Y_red E must equal the generator currents of the augmented network solved
    directly with the internal EMFs as voltage sources."""
    net, sc, r, M = base118
    rng = np.random.default_rng(4)
    E = rng.normal(size=M.m) + 1j * rng.normal(size=M.m)
    nb = net.n_bus
    Y, *_ = grid.ybus(net, sc.br)
    yl = (net.Pd[0] - 1j * net.Qd[0]) / net.base_mva / r["Vm"] ** 2
    ym = 1.0 / (1j * M.xp)
    gb = net.gbus[sc.gen]
    # unknown bus voltages U: (Y + diag(yl)) U + sum_k ym_k (U_gk - E_k) e_gk = 0
    Aug = Y + np.diag(yl)
    rhs = np.zeros(nb, complex)
    for k in range(M.m):
        Aug[gb[k], gb[k]] += ym[k]
        rhs[gb[k]] += ym[k] * E[k]
    U = np.linalg.solve(Aug, rhs)
    I = ym * (E - U[gb])
    assert np.abs(M.Yred @ E - I).max() < 1e-9 * np.abs(I).max()
    assert np.abs(M.Yred - M.Yred.T).max() < 1e-9 * np.abs(M.Yred).max()


def test_generator_outage_shrinks_model():
    net = synth.case118()
    sc = grid.make_scenario(net, 0, net.n_branch + 5)
    r = opf.solve(net, sc)
    assert r["converged"]
    M = dynamics.Model(net, sc, r["Va"], r["Vm"], r["Pg"], r["Qg"])
    assert M.state_matrix().shape == (5 * (net.n_gen - 1),) * 2
    assert M.reduced_state_matrix().shape == (5 * (net.n_gen - 1) - 1,) * 2
