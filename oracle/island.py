"""Main-island OPF of an islanded scenario, with slack re-assignment (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section II-B-3 marks every islanded scenario severe.  Section II-A remarks that,
once a network splits, only the main island (the one tied to the largest
generation) should be taken as reference, and Section V-A traces most of the
study's ~1,390 failed cases to a slack bus that is isolated or inside an
island.  The outlook (Section VI) names the load shed in MW as a non-binary
severity.  This module is the extension that follows those three remarks; the
binary severity of an islanded scenario stays 1.

Readings (the paper gives the idea, not the rules):
  * main island: the connected component whose in-service generators have the
    largest total Pmax (summed in per unit, in generator order); among equal
    totals, the component holding the lowest-numbered bus.  No component with
    a positive total: no main island, the OPF is not run;
  * reference: the original reference bus if it lies in the main island, else
    the bus of the main island's in-service generator with the largest Pmax
    (the lowest generator index among equals);
  * load shed: the active load (MW) of every bus outside the main island;
  * the main island's OPF is the unchanged OPF (``opf.solve``) of the network
    made of the main island alone: its buses renumbered in increasing order,
    the in-service branches and generators inside it, the new reference; a
    point that converges within every limit then gets the unchanged small-signal
    screen (``dynamics``, ``eig``) of that network, whose machines are the main
    island's in-service units (angles referred to the first of them).  Its class
    follows the pipeline's precedence: OPF_NONCONV (2), LIMIT (3), EIG_FAIL (6),
    SS_UNSTABLE (4), SS_POORLY_DAMPED (5) or SECURE (0).  Bus voltages outside
    the main island are reported as 0 (de-energised).

Pins (``tests/test_oracle_island.py``): two networks built apart and joined by
one tie branch; with the tie out, the main island's OPF and small-signal screen
equal the standalone ones of the network with the larger generation (cost,
magnitudes, angles up to the reference shift, class, max Re, min damping ratio),
the shed is the other network's load, and swapping the generation swaps the
choice; a generator outage that reverses the capacities moves the main island to
the side with fewer buses; of three islands the one with the largest capacity
wins; equal generation picks the island of bus 0.
"""
from __future__ import annotations

import copy

import numpy as np

from . import grid, opf, dynamics, eig

SECURE, OPF_NONCONV, LIMIT, SS_UNSTABLE, SS_POORLY_DAMPED, EIG_FAIL = 0, 2, 3, 4, 5, 6
NOT_ISLANDED = 255
DAMPING_MIN = 0.05


def island_labels(n_bus: int, f, t) -> np.ndarray:
    """Component label of every bus, by breadth-first search from the lowest
    unlabelled bus; labels therefore increase with each component's lowest bus."""
    adj = [[] for _ in range(n_bus)]
    for a, b in zip(f, t):
        adj[int(a)].append(int(b))
        adj[int(b)].append(int(a))
    lab = np.full(n_bus, -1, np.int64)
    nxt = 0
    for s in range(n_bus):
        if lab[s] >= 0:
            continue
        lab[s] = nxt
        q = [s]
        while q:
            u = q.pop()
            for w in adj[u]:
                if lab[w] < 0:
                    lab[w] = nxt
                    q.append(w)
        nxt += 1
    return lab


def main_island(net, sc: grid.Scenario):
    """(live bus mask, reference bus, load shed in MW) of scenario sc; the mask is
    None when no component has positive generation capacity."""
    B = net.base_mva
    lab = island_labels(net.n_bus, net.f[sc.br], net.t[sc.br])
    ncomp = int(lab.max()) + 1
    cap = [0.0] * ncomp
    for k in sc.gen:                                   # generator order, per unit
        cap[lab[net.gbus[k]]] += net.Pmax[k] / B
    main, best = -1, 0.0
    for c in range(ncomp):                             # lowest bus first: ties keep the earlier
        if cap[c] > best:
            main, best = c, cap[c]
    Pd = net.Pd[sc.level]
    if main < 0:
        shed = 0.0
        for i in range(net.n_bus):
            shed += Pd[i] / B
        return None, -1, B * shed
    live = lab == main
    if live[net.ref_bus]:
        ref = int(net.ref_bus)
    else:
        kbest, pbest = -1, -np.inf
        for k in sc.gen:
            if live[net.gbus[k]] and net.Pmax[k] / B > pbest:
                kbest, pbest = int(k), net.Pmax[k] / B
        ref = int(net.gbus[kbest])
    shed = 0.0
    for i in range(net.n_bus):
        if not live[i]:
            shed += Pd[i] / B
    return live, ref, B * shed


def sub_network(net, sc: grid.Scenario, live: np.ndarray, ref: int):
    """The main island as a network of its own: live buses renumbered in
    increasing order, the in-service branches and generators inside it."""
    new = np.full(net.n_bus, -1, np.int64)
    new[live] = np.arange(int(live.sum()))
    br = np.array([b for b in sc.br if live[net.f[b]]], np.int64)
    gen = np.array([k for k in sc.gen if live[net.gbus[k]]], np.int64)
    sub = copy.copy(net)
    for name in ("Vmin", "Vmax", "Gs", "Bs", "Pd_shape", "Qd_shape"):
        setattr(sub, name, np.asarray(getattr(net, name))[live].copy())
    sub.Pd = np.asarray(net.Pd)[:, live].copy()
    sub.Qd = np.asarray(net.Qd)[:, live].copy()
    sub.f = new[net.f[br]]
    sub.t = new[net.t[br]]
    for name in ("r", "x", "b", "rate", "tap", "kind"):
        setattr(sub, name, np.asarray(getattr(net, name))[br].copy())
    sub.gbus = new[net.gbus[gen]]
    for name in ("Pmin", "Pmax", "Qmin", "Qmax", "c2", "c1", "c0", "H", "D",
                 "xd", "xq", "xdp", "Td0p", "Tq0p", "KA", "TA"):
        v = getattr(net, name, None)
        if v is not None:
            setattr(sub, name, np.asarray(v)[gen].copy())
    sub.ref_bus = int(new[ref])
    return sub, grid.make_scenario(sub, sc.level)


def evaluate_main_island(net, level: int, i: int = -1, j: int = -1, k: int = -1,
                         damping_min: float = DAMPING_MIN):
    """Main-island result of scenario (level, i, j[, k]).  A scenario that does not
    split gets main_klass NOT_ISLANDED and no OPF (the ordinary path covers it)."""
    sc = grid.make_scenario(net, level, i, j, k)
    nan = float("nan")
    out = dict(main_klass=NOT_ISLANDED, shed_mw=0.0, opf_iters=0, converged=False, cost=nan,
               v_margin=nan, max_loading=nan, max_re=nan, min_zeta=nan, ref=-1, live=None, Va=None, Vm=None)
    if grid.count_islands(net.n_bus, net.f[sc.br], net.t[sc.br]) <= 1:
        return out
    live, ref, shed = main_island(net, sc)
    out.update(shed_mw=shed, main_klass=OPF_NONCONV, ref=ref, live=live)
    if live is None:
        return out
    sub, subsc = sub_network(net, sc, live, ref)
    r = opf.solve(sub, subsc)
    Va = np.zeros(net.n_bus)
    Vm = np.zeros(net.n_bus)
    Va[live] = r["Va"]
    Vm[live] = r["Vm"]
    out.update(opf_iters=r["iterations"], converged=r["converged"], Va=Va, Vm=Vm)
    if not r["converged"]:
        return out
    out["cost"] = r["cost"]
    out["v_margin"], out["max_loading"] = opf.severity_indices(r)
    if opf.limit_violation(r):
        out["main_klass"] = LIMIT
        return out
    model = dynamics.Model(sub, subsc, r["Va"], r["Vm"], r["Pg"], r["Qg"])
    lam, ok, _ = eig.eigvals(model.reduced_state_matrix())
    if not ok:
        out["main_klass"] = EIG_FAIL
        return out
    max_re, min_zeta = eig.stability_stats(lam)
    out.update(max_re=max_re, min_zeta=min_zeta)
    if max_re >= 0.0:
        out["main_klass"] = SS_UNSTABLE
    elif min_zeta < damping_min:
        out["main_klass"] = SS_POORLY_DAMPED
    else:
        out["main_klass"] = SECURE
    return out


# ---- many scenarios in spawned worker processes (tests) ----

_NET = None


def _init_worker(net):
    global _NET
    _NET = net


def _eval_one(args):
    level, i, j = args
    return evaluate_main_island(_NET, level, i, j)


def evaluate_main_island_many(net, scenarios, processes: int | None = None):
    """evaluate_main_island over a list of (level, i, j) in spawned workers (one BLAS
    thread each; spawned, never forked, so it is safe after CUDA use)."""
    import multiprocessing as mp
    import os
    args = [(int(l), int(i), int(j)) for (l, i, j) in scenarios]
    procs = min(processes or os.cpu_count() or 1, max(1, len(args)))
    if procs <= 1:
        _init_worker(net)
        return [_eval_one(a) for a in args]
    old = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in old:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(procs, initializer=_init_worker, initargs=(net,)) as pool:
            return pool.map(_eval_one, args, chunksize=max(1, len(args) // (4 * procs)))
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
