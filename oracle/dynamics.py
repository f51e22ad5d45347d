"""Linearised generator + voltage-regulator model at the OPF point (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section II-B-2 linearises the full system model (generator dynamics and voltage
regulation) at the OPF operating point and inspects the eigenvalues of the
state matrix.  The paper's EMT-based tool is not described; the model used by
the project is written here in its plainest form.

Per in-service generator (machine base S_m = Pmax, converted to system base):

  states         delta, omega, e'q, e'd, Efd     (state index 5k + s)
  EMF            E' = (e'q - j e'd) e^{j delta}   (two-axis, x'd = x'q = x', Ra = 0)
  network        I = Y_red E', Y_red the Kron reduction of the network to the
                 generator internal nodes: loads as constant admittances
                 (Pd - jQd)/|V|^2 at the OPF voltage, each machine an admittance
                 1/(j x') between its internal node and its bus
  dq quantities  i_d + j i_q = j I e^{-j delta},  Pe = e'd i_d + e'q i_q,
                 V_t = E' - j x' I
  equations      d delta/dt = w_s (omega - 1)
                 2H d omega/dt = Pm - Pe - D (omega - 1)
                 T'd0 d e'q/dt = -e'q - (x_d - x') i_d + Efd
                 T'q0 d e'd/dt = -e'd + (x_q - x') i_q
                 T_A d Efd/dt = -Efd + K_A (V_ref - |V_t|)
  equilibrium    from the OPF voltage V and injection Pg + jQg of each machine:
                 I = conj(S/V), delta = arg(V + j x_q I), dq projections,
                 e'q = v_q + x' i_d, e'd = v_d - x' i_q, Efd = e'q + (x_d - x') i_d,
                 V_ref = |V| + Efd/K_A, Pm = Pg, omega = 1.

Angle reference.  With absolute rotor angles and constant-impedance loads a
common rotation of every angle is an equilibrium direction (A v0 = 0 for
v0 = delta-all-ones), so A has one exact zero eigenvalue that carries no
stability information, and the slow common-frequency mode is nearly parallel
to it (eigenvalue condition number ~ w_s / sigma ~ 4e3).  The paper is silent;
the reading used refers every angle to the first in-service machine r:
delta'_k = delta_k - delta_r (k != r) with d delta'_k/dt = w_s (omega_k - omega_r),
and delta_r is dropped.  The reduced matrix A' (5m - 1 states) has exactly the
eigenvalues of A less one zero, and its decisive slow mode is well conditioned.

A = df/dx is obtained by forward-mode automatic differentiation of the state
equations above (a value plus a tangent for every state), so the oracle never
writes a derivative by hand; the CUDA path uses hand-derived derivatives
instead.  Pinned in ``tests/test_oracle_dynamics.py``: A and A' against central
differences with Richardson extrapolation, f(x0) = 0 at the equilibrium,
A v0 = 0 for the common-rotation vector, eig(A') = eig(A) less one zero, and
Y_red against a full nodal solve of the augmented network.
"""
from __future__ import annotations

import numpy as np

from . import grid


class Dual:
    """Vector of values with tangents: v has shape (m,), d has shape (m, n)."""

    __slots__ = ("v", "d")
    __array_ufunc__ = None        # let ndarray (op) Dual defer to Dual's reflected operators

    def __init__(self, v, d):
        self.v = np.asarray(v, dtype=np.float64)
        self.d = np.asarray(d, dtype=np.float64)

    @staticmethod
    def const(v, n):
        v = np.asarray(v, dtype=np.float64)
        return Dual(v, np.zeros(v.shape + (n,)))

    def __add__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v + o.v, self.d + o.d)
        return Dual(self.v + o, self.d)

    __radd__ = __add__

    def __sub__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v - o.v, self.d - o.d)
        return Dual(self.v - o, self.d)

    def __rsub__(self, o):
        return Dual(o - self.v, -self.d)

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __mul__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v * o.v, self.d * o.v[:, None] + o.d * self.v[:, None])
        o = np.asarray(o, dtype=np.float64)
        return Dual(self.v * o, self.d * (o[:, None] if o.ndim else o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v / o.v, (self.d * o.v[:, None] - o.d * self.v[:, None]) / (o.v ** 2)[:, None])
        o = np.asarray(o, dtype=np.float64)
        return Dual(self.v / o, self.d / (o[:, None] if o.ndim else o))

    def matmul_left(self, M):
        """M @ self for a constant matrix M."""
        return Dual(M @ self.v, M @ self.d)


def dsin(x: Dual) -> Dual:
    return Dual(np.sin(x.v), np.cos(x.v)[:, None] * x.d)


def dcos(x: Dual) -> Dual:
    return Dual(np.cos(x.v), -np.sin(x.v)[:, None] * x.d)


def dsqrt(x: Dual) -> Dual:
    r = np.sqrt(x.v)
    return Dual(r, x.d / (2.0 * r)[:, None])


class Model:
    """Small-signal model of one scenario at a converged OPF point."""

    def __init__(self, net, sc: grid.Scenario, Va, Vm, Pg, Qg):
        B = net.base_mva
        g = sc.gen
        self.m = m = len(g)
        self.gen = g
        Sm = net.Pmax[g]
        zb = B / Sm                               # machine -> system impedance factor
        self.xd = net.xd[g] * zb
        self.xq = net.xq[g] * zb
        self.xp = net.xdp[g] * zb
        self.Td0 = net.Td0p[g]
        self.Tq0 = net.Tq0p[g]
        self.KA = net.KA[g]
        self.TA = net.TA[g]
        self.H = net.H[g] * Sm / B
        self.D = net.D[g] * Sm / B
        self.ws = 2.0 * np.pi * net.f_hz

        V = Vm * np.exp(1j * Va)
        Y, _, _, _, _ = grid.ybus(net, sc.br)
        Pd = net.Pd[sc.level] / B
        Qd = net.Qd[sc.level] / B
        yl = (Pd - 1j * Qd) / (Vm ** 2)
        ym = 1.0 / (1j * self.xp)
        nb = net.n_bus
        gb = net.gbus[g]
        Ybb = Y + np.diag(yl)
        Ybg = np.zeros((nb, m), complex)
        for k in range(m):
            Ybb[gb[k], gb[k]] += ym[k]
            Ybg[gb[k], k] = -ym[k]
        Ygg = np.diag(ym)
        self.Yred = Ygg - Ybg.T @ np.linalg.solve(Ybb, Ybg)

        # equilibrium
        Vt = V[gb]
        S = Pg + 1j * Qg
        I = np.conj(S / Vt)
        EQ = Vt + 1j * self.xq * I
        delta = np.angle(EQ)
        rot = 1j * np.exp(-1j * delta)           # network frame -> dq frame
        Idq = I * rot
        Vdq = Vt * rot
        i_d, i_q = Idq.real, Idq.imag
        v_d, v_q = Vdq.real, Vdq.imag
        eq = v_q + self.xp * i_d
        ed = v_d - self.xp * i_q
        Efd = eq + (self.xd - self.xp) * i_d
        self.Vref = np.abs(Vt) + Efd / self.KA
        self.Pm = Pg.copy()
        x0 = np.zeros(5 * m)
        x0[0::5] = delta
        x0[1::5] = 1.0
        x0[2::5] = eq
        x0[3::5] = ed
        x0[4::5] = Efd
        self.x0 = x0

    def f(self, x: Dual) -> Dual:
        """State derivatives (as a Dual); x is a Dual over the 5m states."""
        m = self.m
        n = x.d.shape[1]

        def pick(s):
            return Dual(x.v[s::5], x.d[s::5])

        delta, omega, eq, ed, Efd = (pick(s) for s in range(5))
        c, s = dcos(delta), dsin(delta)
        Er = eq * c + ed * s                      # Re E'
        Ei = eq * s - ed * c                      # Im E'
        G, Bm = self.Yred.real, self.Yred.imag
        Ir = Er.matmul_left(G) - Ei.matmul_left(Bm)
        Ii = Er.matmul_left(Bm) + Ei.matmul_left(G)
        i_d = Ir * s - Ii * c
        i_q = Ir * c + Ii * s
        Pe = ed * i_d + eq * i_q
        Vr = Er + Ii * self.xp
        Vi = Ei - Ir * self.xp
        Vt = dsqrt(Vr * Vr + Vi * Vi)
        out_v = np.zeros(5 * m)
        out_d = np.zeros((5 * m, n))
        rows = [
            (omega - 1.0) * self.ws,
            (self.Pm - Pe - (omega - 1.0) * self.D) / (2.0 * self.H),
            (-eq - i_d * (self.xd - self.xp) + Efd) / self.Td0,
            (-ed + i_q * (self.xq - self.xp)) / self.Tq0,
            (-Efd + (self.Vref - Vt) * self.KA) / self.TA,
        ]
        for k, r in enumerate(rows):
            out_v[k::5] = r.v
            out_d[k::5] = r.d
        return Dual(out_v, out_d)

    def f_value(self, xv):
        return self.f(Dual(xv, np.zeros((xv.size, 1)))).v

    def state_matrix(self):
        """A = df/dx over the absolute states (5m)."""
        n = 5 * self.m
        return self.f(Dual(self.x0, np.eye(n))).d

    def reduced_state_matrix(self):
        """A' over the states with angles referred to machine 0 (5m - 1):
        reduced index 5k + s - 1 for every state but delta_0."""
        m = self.m
        nf, nr = 5 * m, 5 * m - 1
        val = self.x0.copy()
        tan = np.zeros((nf, nr))
        for i in range(1, nf):
            tan[i, i - 1] = 1.0
        for k in range(1, m):
            tan[5 * k, :] = 0.0
            tan[5 * k, 5 * k - 1] = 1.0     # delta_k = delta_0 (constant) + delta'_k
        f = self.f(Dual(val, tan)).d
        out = f[1:].copy()                  # drop the delta_0 row
        for k in range(1, m):
            out[5 * k - 1] = f[5 * k] - f[0]   # d delta'_k / dt = f_delta_k - f_delta_0
        return out
