"""Primal-dual interior-point AC optimal power flow (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section II-B-1: a contingency is severe when the AC OPF does not converge, or
when its converged solution violates an operational limit.  The paper delegates
the OPF to an external tool and states no algorithm; this module implements the
reading used throughout the project: the MIPS primal-dual interior-point method
(Wang, Murillo-Sanchez, Zimmerman and Thomas, IEEE Trans. Power Syst. 2007) in
polar voltage coordinates, written densely and serially:

  variables      x = [Va (nb), Vm (nb), Pg (ng), Qg (ng)]   (per unit, rad)
  cost           f = sum c2 (B Pg)^2 + c1 (B Pg) + c0        (B = base MVA, $/h)
  equalities     g = [Re S(V) - Cg Pg + Pd ; Im S(V) - Cg Qg + Qd ; Va_ref]
  inequalities   h = [|S_f|^2 - Smax^2 ; |S_t|^2 - Smax^2 ;
                      Vm - Vmax ; Vmin - Vm ; Pg - Pmax ; Pmin - Pg ;
                      Qg - Qmax ; Qmin - Qg]
  start          Va = 0, Vm = 1, Pg = (Pmin + Pmax)/2, Qg = 0,
                 z = max(-h, 1), gamma = 1, mu = gamma / z, lam = 0
  Newton system  [M, Jg^T; Jg, 0] [dx; dlam] = -[N; g],
                 M = Lxx + Jh^T diag(mu/z) Jh,  N = Lx + Jh^T diag(1/z)(mu*h + gamma)
                 dz = -h - z - Jh dx,  dmu = -mu + (gamma - mu*dz)/z
  step           alpha_p = min(xi min_{dz<0} -z/dz, 1), alpha_d likewise on mu,
                 xi = 0.99995; gamma = sigma z^T mu / n_in, sigma = 0.1
  stop           feasibility, gradient, complementarity and cost-change
                 conditions all below tol (1e-8), at most 50 iterations;
                 any non-finite value or a singular Newton matrix = no convergence.

The Newton matrix is solved with a dense LU with partial pivoting
(``numpy.linalg.solve``) on the full, unreduced system.

The derivatives are this module's own derivation.  With V = Vm e^{j Va}, every
power-flow quantity used here has the form Re(sum_ik W_ik V_i conj(V_k)) for a
constant complex matrix W; ``quad_hessian`` gives its exact Hessian with respect
to (Va, Vm).  Pinned in ``tests/test_oracle_opf.py`` against central finite
differences, the two-bus power-flow closed form, the two-generator lossless
economic dispatch closed form and the KKT residuals at every converged point.
``conditions`` is pinned against values worked by hand from the MIPS
definitions, and the stopping rule against the iteration trace;
``limit_violation`` against limits moved across a converged two-bus point whose
flow is computed from its voltages alone (violated beyond 1e-6 p.u., not within).
"""
from __future__ import annotations

import numpy as np

from . import grid

TOL = 1e-8
MAX_IT = 50
XI = 0.99995
SIGMA = 0.1
LIMIT_TOL = 1e-6


def quad_hessian(W, V, Vm):
    """Hessian w.r.t. (Va, Vm) of Re(sum_ik W_ik V_i conj(V_k)), V = Vm e^{jVa}."""
    Wc = W @ np.conj(V)
    WtV = W.T @ V
    D = {0: 1j * V, 1: V / Vm}
    d2 = {(0, 0): -V, (0, 1): 1j * V / Vm, (1, 0): 1j * V / Vm, (1, 1): np.zeros_like(V)}
    nb = V.shape[0]
    H = np.zeros((2 * nb, 2 * nb))
    for p in (0, 1):
        for q in (0, 1):
            blk = (np.diag(d2[p, q] * Wc)
                   + D[p][:, None] * W * np.conj(D[q])[None, :]
                   + (D[q][:, None] * W * np.conj(D[p])[None, :]).T
                   + np.diag(np.conj(d2[p, q]) * WtV))
            H[p * nb:(p + 1) * nb, q * nb:(q + 1) * nb] = blk.real
    return H


def _dS(Cx, Yx, V, Vm):
    """Jacobians of S_x = (Cx V) conj(Yx V) w.r.t. Va and Vm (complex, rows = Cx rows)."""
    Ix = Yx @ V
    Vx = Cx @ V
    dVa = 1j * V
    dVm = V / Vm
    dS_dVa = np.conj(Ix)[:, None] * Cx * dVa[None, :] + Vx[:, None] * np.conj(Yx * dVa[None, :])
    dS_dVm = np.conj(Ix)[:, None] * Cx * dVm[None, :] + Vx[:, None] * np.conj(Yx * dVm[None, :])
    return Vx * np.conj(Ix), dS_dVa, dS_dVm


class Problem:
    """The OPF of one scenario: data of the network with outaged elements removed."""

    def __init__(self, net, sc: grid.Scenario):
        B = net.base_mva
        self.B = B
        self.nb = nb = net.n_bus
        self.br = sc.br
        self.gen = sc.gen
        self.ng = ng = len(sc.gen)
        self.nl = nl = len(sc.br)
        self.ref = net.ref_bus
        self.Y, self.Yf, self.Yt, self.Cf, self.Ct = grid.ybus(net, sc.br)
        self.Ib = np.eye(nb)
        self.Cg = np.zeros((nb, ng))
        self.Cg[net.gbus[sc.gen], np.arange(ng)] = 1.0
        self.Pd = net.Pd[sc.level] / B
        self.Qd = net.Qd[sc.level] / B
        self.Smax2 = (net.rate[sc.br] / B) ** 2
        self.Vmin, self.Vmax = net.Vmin.copy(), net.Vmax.copy()
        g = sc.gen
        self.Pmin, self.Pmax = net.Pmin[g] / B, net.Pmax[g] / B
        self.Qmin, self.Qmax = net.Qmin[g] / B, net.Qmax[g] / B
        self.c2, self.c1, self.c0 = net.c2[g], net.c1[g], net.c0[g]
        self.nx = 2 * nb + 2 * ng
        self.neq = 2 * nb + 1
        self.niq = 2 * nl + 2 * nb + 4 * ng

    def x0(self):
        nb, ng = self.nb, self.ng
        x = np.zeros(self.nx)
        x[nb:2 * nb] = 1.0
        x[2 * nb:2 * nb + ng] = 0.5 * (self.Pmin + self.Pmax)
        return x

    def split(self, x):
        nb, ng = self.nb, self.ng
        return x[:nb], x[nb:2 * nb], x[2 * nb:2 * nb + ng], x[2 * nb + ng:]

    def evaluate(self, x):
        """f, grad f, g, h, Jg, Jh and the pieces the Hessian needs."""
        nb, ng, nl, B = self.nb, self.ng, self.nl, self.B
        Va, Vm, Pg, Qg = self.split(x)
        V = Vm * np.exp(1j * Va)
        PgMW = B * Pg
        f = float(np.sum(self.c2 * PgMW ** 2 + self.c1 * PgMW + self.c0))
        df = np.zeros(self.nx)
        df[2 * nb:2 * nb + ng] = B * (2.0 * self.c2 * PgMW + self.c1)

        Sb, dSb_dVa, dSb_dVm = _dS(self.Ib, self.Y, V, Vm)
        Sf, dSf_dVa, dSf_dVm = _dS(self.Cf, self.Yf, V, Vm)
        St, dSt_dVa, dSt_dVm = _dS(self.Ct, self.Yt, V, Vm)

        g = np.concatenate([Sb.real - self.Cg @ Pg + self.Pd,
                            Sb.imag - self.Cg @ Qg + self.Qd,
                            [Va[self.ref]]])
        Jg = np.zeros((self.neq, self.nx))
        Jg[:nb, :nb] = dSb_dVa.real
        Jg[:nb, nb:2 * nb] = dSb_dVm.real
        Jg[:nb, 2 * nb:2 * nb + ng] = -self.Cg
        Jg[nb:2 * nb, :nb] = dSb_dVa.imag
        Jg[nb:2 * nb, nb:2 * nb] = dSb_dVm.imag
        Jg[nb:2 * nb, 2 * nb + ng:] = -self.Cg
        Jg[2 * nb, self.ref] = 1.0

        h = np.concatenate([np.abs(Sf) ** 2 - self.Smax2, np.abs(St) ** 2 - self.Smax2,
                            Vm - self.Vmax, self.Vmin - Vm,
                            Pg - self.Pmax, self.Pmin - Pg,
                            Qg - self.Qmax, self.Qmin - Qg])
        Jh = np.zeros((self.niq, self.nx))
        Jh[:nl, :nb] = 2.0 * (np.conj(Sf)[:, None] * dSf_dVa).real
        Jh[:nl, nb:2 * nb] = 2.0 * (np.conj(Sf)[:, None] * dSf_dVm).real
        Jh[nl:2 * nl, :nb] = 2.0 * (np.conj(St)[:, None] * dSt_dVa).real
        Jh[nl:2 * nl, nb:2 * nb] = 2.0 * (np.conj(St)[:, None] * dSt_dVm).real
        r = 2 * nl
        I = np.eye(nb)
        Jh[r:r + nb, nb:2 * nb] = I
        Jh[r + nb:r + 2 * nb, nb:2 * nb] = -I
        r += 2 * nb
        Ig = np.eye(ng)
        Jh[r:r + ng, 2 * nb:2 * nb + ng] = Ig
        Jh[r + ng:r + 2 * ng, 2 * nb:2 * nb + ng] = -Ig
        r += 2 * ng
        Jh[r:r + ng, 2 * nb + ng:] = Ig
        Jh[r + ng:r + 2 * ng, 2 * nb + ng:] = -Ig
        cache = dict(V=V, Vm=Vm, Sf=Sf, St=St, dSf=(dSf_dVa, dSf_dVm), dSt=(dSt_dVa, dSt_dVm))
        return f, df, g, h, Jg, Jh, cache

    def hessian(self, cache, lam, mu):
        """Hessian of the Lagrangian f + lam^T g + mu^T h."""
        nb, ng, nl, B = self.nb, self.ng, self.nl, self.B
        V, Vm = cache["V"], cache["Vm"]
        Lxx = np.zeros((self.nx, self.nx))
        lamP, lamQ = lam[:nb], lam[nb:2 * nb]
        W = (lamP - 1j * lamQ)[:, None] * np.conj(self.Y)
        Hv = quad_hessian(W, V, Vm)
        for (S, dS, C, Yx, m) in ((cache["Sf"], cache["dSf"], self.Cf, self.Yf, mu[:nl]),
                                  (cache["St"], cache["dSt"], self.Ct, self.Yt, mu[nl:2 * nl])):
            Wx = C.T @ ((2.0 * m * np.conj(S))[:, None] * np.conj(Yx))
            Hv += quad_hessian(Wx, V, Vm)
            dSv = np.hstack([dS[0], dS[1]])
            Hv += 2.0 * (np.conj(dSv).T @ (m[:, None] * dSv)).real
        Lxx[:2 * nb, :2 * nb] = Hv
        idx = np.arange(2 * nb, 2 * nb + ng)
        Lxx[idx, idx] = 2.0 * self.c2 * B * B
        return Lxx


def conditions(prob, x, z, lam, mu, f, f_prev, g, h, Lx):
    """The four MIPS stopping quantities."""
    nx_inf = np.max(np.abs(x)) if x.size else 0.0
    feas = max(np.max(np.abs(g)), np.max(h)) / (1.0 + max(nx_inf, np.max(np.abs(z))))
    grad = np.max(np.abs(Lx)) / (1.0 + max(np.max(np.abs(lam)), np.max(np.abs(mu))))
    comp = float(z @ mu) / (1.0 + nx_inf)
    cost = abs(f - f_prev) / (1.0 + abs(f_prev))
    return feas, grad, comp, cost


def solve(net, sc: grid.Scenario, tol=TOL, max_it=MAX_IT, xi=XI, sigma=SIGMA, trace=False):
    """Run the interior-point OPF of one scenario.  Returns a dict with
    ``converged``, ``iterations``, ``cost`` and the primal/dual point."""
    prob = Problem(net, sc)
    x = prob.x0()
    f, df, g, h, Jg, Jh, cache = prob.evaluate(x)
    gamma = 1.0
    lam = np.zeros(prob.neq)
    z = np.maximum(-h, 1.0)
    mu = gamma / z
    Lx = df + Jg.T @ lam + Jh.T @ mu
    f_prev = f
    hist = []
    conds = conditions(prob, x, z, lam, mu, f, f_prev, g, h, Lx)
    converged = all(c < tol for c in conds)
    it = 0
    failed = False
    while not converged and it < max_it:
        it += 1
        Lxx = prob.hessian(cache, lam, mu)
        zinv = 1.0 / z
        M = Lxx + Jh.T @ ((mu * zinv)[:, None] * Jh)
        N = Lx + Jh.T @ (zinv * (mu * h + gamma))
        K = np.block([[M, Jg.T], [Jg, np.zeros((prob.neq, prob.neq))]])
        rhs = -np.concatenate([N, g])
        try:
            sol = np.linalg.solve(K, rhs)
        except np.linalg.LinAlgError:
            failed = True
            break
        if not np.all(np.isfinite(sol)):
            failed = True
            break
        dx, dlam = sol[:prob.nx], sol[prob.nx:]
        dz = -h - z - Jh @ dx
        dmu = -mu + zinv * (gamma - mu * dz)
        k = dz < 0
        alpha_p = min(xi * np.min(-z[k] / dz[k]), 1.0) if np.any(k) else 1.0
        k = dmu < 0
        alpha_d = min(xi * np.min(-mu[k] / dmu[k]), 1.0) if np.any(k) else 1.0
        x = x + alpha_p * dx
        z = z + alpha_p * dz
        lam = lam + alpha_d * dlam
        mu = mu + alpha_d * dmu
        gamma = sigma * float(z @ mu) / prob.niq
        f_prev = f
        f, df, g, h, Jg, Jh, cache = prob.evaluate(x)
        Lx = df + Jg.T @ lam + Jh.T @ mu
        if not (np.all(np.isfinite(x)) and np.isfinite(f) and np.all(np.isfinite(lam))
                and np.all(np.isfinite(mu)) and np.all(np.isfinite(z))):
            failed = True
            break
        conds = conditions(prob, x, z, lam, mu, f, f_prev, g, h, Lx)
        if trace:
            hist.append((it, alpha_p, alpha_d, gamma) + tuple(conds))
        converged = all(c < tol for c in conds)
    converged = converged and not failed
    Va, Vm, Pg, Qg = prob.split(x)
    return dict(converged=bool(converged), iterations=it, failed=failed, cost=f,
                Va=Va.copy(), Vm=Vm.copy(), Pg=Pg.copy(), Qg=Qg.copy(),
                lam=lam, mu=mu, z=z, h=h, g=g, Lx=Lx, conds=conds, hist=hist, prob=prob)


def severity_indices(res):
    """Non-binary severity of a converged point (an extension the paper names in its
    outlook, Section VI): the smallest voltage margin min_i min(Vm_i - Vmin_i,
    Vmax_i - Vm_i) in p.u., and the largest branch loading max |S| / Smax over both
    ends of the in-service branches."""
    prob = res["prob"]
    Vm = res["Vm"]
    nl = prob.nl
    h = res["h"]
    smax = np.sqrt(prob.Smax2)
    sf = np.sqrt(np.maximum(h[:nl] + prob.Smax2, 0.0))
    st = np.sqrt(np.maximum(h[nl:2 * nl] + prob.Smax2, 0.0))
    margin = float(min(np.min(Vm - prob.Vmin), np.min(prob.Vmax - Vm)))
    loading = float(max(np.max(sf / smax), np.max(st / smax))) if nl else 0.0
    return margin, loading


def limit_violation(res, tol=LIMIT_TOL) -> bool:
    """Section II-B-1 operational limits at a converged point: thermal (|S| above
    Smax) and voltage / generator bounds, each beyond ``tol`` per unit."""
    prob = res["prob"]
    h = res["h"]
    nl = prob.nl
    Smax = np.sqrt(prob.Smax2)
    Sf = np.sqrt(np.maximum(h[:nl] + prob.Smax2, 0.0))
    St = np.sqrt(np.maximum(h[nl:2 * nl] + prob.Smax2, 0.0))
    if np.any(Sf - Smax > tol) or np.any(St - Smax > tol):
        return True
    return bool(np.any(h[2 * nl:] > tol))
