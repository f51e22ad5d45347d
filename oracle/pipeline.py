"""One contingency scenario end to end, and its severity class (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section II-A enumerates scenarios (base, every single outage i, every pair);
Section II-B decides the binary severity S_c from three criteria.  Order of
the checks here: islanding first (an OPF on a split network is what produced
the paper's numerical failures, Section V-A), then the OPF and its limit check,
then the eigenvalue screen of the linearised model.  The class records the
first criterion that failed; S_c = 1 for every class but SECURE.

Classes: SECURE 0, ISLANDED 1, OPF_NONCONV 2, LIMIT 3, SS_UNSTABLE 4
(max Re >= 0 of the angle-referenced state matrix), SS_POORLY_DAMPED 5
(minimum damping ratio below ``damping_min``; 0 gives the paper's literal rule,
the study configuration uses 0.05), EIG_FAIL 6 (QR did not converge).
"""
from __future__ import annotations

import os

import numpy as np

from . import grid, opf, dynamics, eig

SECURE, ISLANDED, OPF_NONCONV, LIMIT, SS_UNSTABLE, SS_POORLY_DAMPED, EIG_FAIL = range(7)
DAMPING_MIN = 0.05


def evaluate(net, level: int, i: int = -1, j: int = -1, damping_min: float = DAMPING_MIN,
             keep_state: bool = False, k: int = -1):
    """Evaluate scenario (level, i, j[, k]).  Returns a dict of plain values."""
    sc = grid.make_scenario(net, level, i, j, k)
    nisl = grid.count_islands(net.n_bus, net.f[sc.br], net.t[sc.br])
    out = dict(level=level, i=i, j=j, n_islands=nisl, opf_iters=0, converged=False,
               cost=np.nan, max_re=np.nan, min_zeta=np.nan, eig_sweeps=0, v_margin=np.nan, max_loading=np.nan)
    if nisl > 1:
        out["klass"] = ISLANDED
        out["severe"] = 1
        return out
    r = opf.solve(net, sc)
    out.update(opf_iters=r["iterations"], converged=r["converged"], cost=r["cost"],
               Va=r["Va"], Vm=r["Vm"], Pg=r["Pg"], Qg=r["Qg"], conds=r["conds"])
    if not r["converged"]:
        out["klass"] = OPF_NONCONV
        out["severe"] = 1
        return out
    out["v_margin"], out["max_loading"] = opf.severity_indices(r)
    if opf.limit_violation(r):
        out["klass"] = LIMIT
        out["severe"] = 1
        return out
    model = dynamics.Model(net, sc, r["Va"], r["Vm"], r["Pg"], r["Qg"])
    A = model.reduced_state_matrix()
    lam, ok, sweeps = eig.eigvals(A)
    out["eig_sweeps"] = sweeps
    if keep_state:
        out["A"] = A
        out["eigs"] = lam
        out["model"] = model
    if not ok:
        out["klass"] = EIG_FAIL
        out["severe"] = 1
        return out
    max_re, min_zeta = eig.stability_stats(lam)
    out.update(max_re=max_re, min_zeta=min_zeta)
    if max_re >= 0.0:
        k = SS_UNSTABLE
    elif min_zeta < damping_min:
        k = SS_POORLY_DAMPED
    else:
        k = SECURE
    out["klass"] = k
    out["severe"] = int(k != SECURE)
    return out


# ---- many scenarios in worker processes (used by tests and the CPU baseline) ----

_NET = None


def _init_worker(net):
    global _NET
    _NET = net


def _eval_one(args):
    level, i, j, damping_min = args
    r = evaluate(_NET, level, i, j, damping_min)
    return {k: r[k] for k in ("level", "i", "j", "klass", "severe", "n_islands", "opf_iters",
                              "converged", "cost", "max_re", "min_zeta")} | (
        {"Vm": r["Vm"], "Va": r["Va"]} if "Vm" in r else {})


def evaluate_many(net, scenarios, processes: int | None = None, damping_min: float = DAMPING_MIN):
    """Evaluate a list of (level, i, j) in ``processes`` spawned workers (one
    BLAS thread each).  Spawned, never forked, so it is safe after CUDA use."""
    import multiprocessing as mp
    args = [(int(l), int(i), int(j), damping_min) for (l, i, j) in scenarios]
    procs = processes or os.cpu_count() or 1
    if procs <= 1 or len(args) <= 1:
        _init_worker(net)
        return [_eval_one(a) for a in args]
    old = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in old:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(procs, initializer=_init_worker, initargs=(net,)) as pool:
            return pool.map(_eval_one, args, chunksize=max(1, len(args) // (4 * procs)))
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
