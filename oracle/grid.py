"""Post-contingency network: admittance matrices and island count (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Outaged branches and generators are physically removed here.  Section II-A
(enumeration), Section II-B-3 (islanding: a depth-first-like search counts the
connected subgraphs; more than one island is a failure of maximum severity).

Pins: ``tests/test_oracle_grid.py`` (brute force over all edge subsets of small
graphs, bridges and two-edge cuts found by exhaustive deletion, Ybus row sums
against the shunt-only closed form).
"""
from __future__ import annotations

from collections import deque
from dataclasses import dataclass
import numpy as np


@dataclass
class Scenario:
    """In-service sets of one contingency at one load level."""
    level: int
    out_elems: tuple          # element ids removed (branches first, then generators)
    br: np.ndarray            # indices of in-service branches
    gen: np.ndarray           # indices of in-service generators


def make_scenario(net, level: int, i: int = -1, j: int = -1, k: int = -1) -> Scenario:
    """Scenario with elements i, j and k out (-1 = none; k gives the N-3 extension of
    the enumeration, a repeated id counts once).  Element ids: [0, n_branch) are
    branches, [n_branch, n_branch + n_gen) generators (Section II-A)."""
    out = tuple(sorted({e for e in (i, j, k) if e >= 0}))
    for e in out:
        if e >= net.n_elem:
            raise ValueError("element id out of range")
    br_out = {e for e in out if e < net.n_branch}
    g_out = {e - net.n_branch for e in out if e >= net.n_branch}
    br = np.array([k for k in range(net.n_branch) if k not in br_out], dtype=np.int64)
    gen = np.array([k for k in range(net.n_gen) if k not in g_out], dtype=np.int64)
    return Scenario(level, out, br, gen)


def count_islands(n_bus: int, f, t) -> int:
    """Number of connected components of the bus graph (every bus counts, an
    isolated bus is an island of its own), by breadth-first search."""
    adj = [[] for _ in range(n_bus)]
    for a, b in zip(f, t):
        adj[int(a)].append(int(b))
        adj[int(b)].append(int(a))
    seen = [False] * n_bus
    comps = 0
    for s in range(n_bus):
        if seen[s]:
            continue
        comps += 1
        seen[s] = True
        q = deque([s])
        while q:
            u = q.popleft()
            for w in adj[u]:
                if not seen[w]:
                    seen[w] = True
                    q.append(w)
    return comps


def branch_admittances(net, br):
    """Pi-model two-port admittances of the given branches, per unit:
    I_f = yff V_f + yft V_t, I_t = ytf V_f + ytt V_t (tap ratio on the from side)."""
    ys = 1.0 / (net.r[br] + 1j * net.x[br])
    bc = net.b[br]
    tap = net.tap[br]
    ytt = ys + 0.5j * bc
    yff = ytt / (tap * tap)
    yft = -ys / tap
    ytf = -ys / tap
    return yff, yft, ytf, ytt


def ybus(net, br):
    """Dense bus admittance matrix and the from/to branch admittance matrices
    (rows = in-service branches) of the network with only branches ``br``."""
    nb = net.n_bus
    nl = len(br)
    yff, yft, ytf, ytt = branch_admittances(net, br)
    f = net.f[br].astype(np.int64)
    t = net.t[br].astype(np.int64)
    Cf = np.zeros((nl, nb))
    Ct = np.zeros((nl, nb))
    Cf[np.arange(nl), f] = 1.0
    Ct[np.arange(nl), t] = 1.0
    Yf = np.zeros((nl, nb), complex)
    Yt = np.zeros((nl, nb), complex)
    Yf[np.arange(nl), f] += yff
    Yf[np.arange(nl), t] += yft
    Yt[np.arange(nl), f] += ytf
    Yt[np.arange(nl), t] += ytt
    Ysh = (net.Gs + 1j * net.Bs) / net.base_mva
    Y = Cf.T @ Yf + Ct.T @ Yt + np.diag(Ysh)
    return Y, Yf, Yt, Cf, Ct
