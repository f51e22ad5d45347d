"""Rounding-level variants of the oracle's Newton-step solve.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section II-B runs an interior-point OPF per scenario; each iteration takes the
Newton step, the solution of the KKT system that ``opf.solve`` forms and hands
to ``numpy.linalg.solve``.  Near the optimum the barrier terms of the active
bounds grow like 1/z and the system's condition number passes 1e20 (1e25-1e30
in the last iterations of degenerate scenarios), so its FP64 solution is
decided by rounding: two backward-stable solvers return steps that differ in
their leading digits.  Mostly the differences lie in directions the method
does not care about and the outcome (converged or not, iteration count) is the
same; in a few degenerate scenarios it is not.  The method itself (exact Newton
steps) does not fix the FP64 outcome of such a scenario.

``outcomes`` re-runs the oracle's pipeline on one scenario with each of these
solves of the same system, all backward stable:

* ``lu``: the oracle's own (LAPACK LU with partial pivoting);
* ``ldl``: symmetric indefinite LDL^T with Bunch-Kaufman pivoting (LAPACK);
* ``perm0`` .. ``perm23``: LU of P K P^T for seeded random permutations P;
* ``refined``: LU followed by iterative refinement whose residuals are computed
  exactly and rounded once (Dekker's two-product with Veltkamp splitting, then
  ``math.fsum``), the FP64 rounding of the exact Newton step wherever the
  refinement converges.

A scenario is rounding-decided when the outcomes differ.  Nothing here edits
``opf.py``: inside ``newton_solve`` each OPF runs with the variant in place of
``numpy.linalg.solve`` (its only linear solve), restored when the OPF returns.
"""
from __future__ import annotations

import math
from contextlib import contextmanager

import numpy as np
import scipy.linalg as sla

from . import opf, pipeline

_SPLIT = 134217729.0          # 2^27 + 1, Veltkamp's splitting constant for FP64


def two_product(a, b):
    """p, e with p = fl(a b) and p + e = a b exactly (Dekker), elementwise.
    Exact while |a|, |b| < 2^996 and no product underflows."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    p = a * b
    t = _SPLIT * a
    ah = t - (t - a)
    al = a - ah
    t = _SPLIT * b
    bh = t - (t - b)
    bl = b - bh
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def exact_residual(K, x, b):
    """r = b - K x with every entry the correctly rounded value of the exact sum."""
    K = np.asarray(K, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    p, e = two_product(K, x[None, :])
    r = np.empty(K.shape[0])
    for i in range(K.shape[0]):
        r[i] = math.fsum([float(b[i])] + (-p[i]).tolist() + (-e[i]).tolist())
    return r


def refined_solve(K, rhs, steps: int = 10):
    """LU solution refined with exactly rounded residuals until the correction
    stops shrinking (or ``steps`` corrections)."""
    lu = sla.lu_factor(K, check_finite=False)
    x = sla.lu_solve(lu, rhs, check_finite=False)
    prev = np.inf
    for _ in range(steps):
        d = sla.lu_solve(lu, exact_residual(K, x, rhs), check_finite=False)
        nd = float(np.max(np.abs(d))) if d.size else 0.0
        if not nd < prev:
            break
        x = x + d
        prev = nd
        if nd <= 2.220446049250313e-16 * float(np.max(np.abs(x))):
            break
    return x


def _perm_solver(seed: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    lin = np.linalg.solve

    def solve(K, rhs):
        p = rng.permutation(K.shape[0])
        y = lin(K[np.ix_(p, p)], rhs[p])
        x = np.empty_like(y)
        x[p] = y
        return x
    return solve


N_PERM = 24


def _ldl_solve(K, rhs):
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", sla.LinAlgWarning)      # ill-conditioned by nature here
        return sla.solve(K, rhs, assume_a="sym")


def solver(name: str):
    """solve(K, rhs) of one variant (a fresh permutation generator per call)."""
    if name == "lu":
        return np.linalg.solve
    if name == "ldl":
        return _ldl_solve
    if name == "refined":
        return refined_solve
    if name.startswith("perm") and 0 <= int(name[4:]) < N_PERM:
        return _perm_solver(int(name[4:]))
    raise KeyError(name)


def names() -> list:
    return ["lu", "ldl", "refined"] + [f"perm{k}" for k in range(N_PERM)]


@contextmanager
def newton_solve(fn):
    """Inside the block, every opf.solve takes its Newton steps with fn (the OPF's
    only call of numpy.linalg.solve); the rest of the pipeline is untouched."""
    plain = opf.solve

    def solve_with(*args, **kw):
        lin = np.linalg.solve
        np.linalg.solve = fn
        try:
            return plain(*args, **kw)
        finally:
            np.linalg.solve = lin
    opf.solve = solve_with
    try:
        yield
    finally:
        opf.solve = plain


def _one(args):
    net, level, i, j, name = args
    with newton_solve(solver(name)):
        r = pipeline.evaluate(net, level, i, j)
    return name, (int(r["klass"]), int(r["opf_iters"]))


def outcomes(net, level: int, i: int = -1, j: int = -1, which=None, processes: int = 0) -> dict:
    """name -> (klass, opf_iters) of the oracle pipeline on one scenario under each
    variant (all of them unless ``which``).  processes > 1 runs them in a pool of
    spawned workers (safe in a process that already holds a GPU context)."""
    todo = [(net, level, i, j, n) for n in (which or names())]
    if processes and processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(processes, len(todo))) as pool:
            return dict(pool.map(_one, todo))
    return dict(_one(t) for t in todo)


def rounding_decided(outs: dict) -> bool:
    """True when the variants do not agree on the outcome."""
    return len(set(outs.values())) > 1
