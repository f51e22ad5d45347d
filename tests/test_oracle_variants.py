"""Pins of oracle/variants.py: the exactly rounded residual against rational
arithmetic, the refined solve against the exact solution of an ill-conditioned
system, every variant against the oracle's own solve on scenarios whose Newton
systems are well conditioned, and one 118-bus scenario whose outcome FP64
rounding decides (Section II-B's OPF; the variants solve the same KKT systems)."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2512_08465_gb300 import synth
from oracle import opf, pipeline, variants


def test_two_product_is_exact():
    rng = np.random.default_rng(7)
    a = rng.standard_normal(200) * 10.0 ** rng.integers(-20, 20, 200)
    b = rng.standard_normal(200) * 10.0 ** rng.integers(-20, 20, 200)
    p, e = variants.two_product(a, b)
    for q in range(200):
        assert Fraction(p[q]) + Fraction(e[q]) == Fraction(a[q]) * Fraction(b[q])


def test_exact_residual_is_the_rounded_exact_value():
    rng = np.random.default_rng(11)
    n = 12
    K = rng.standard_normal((n, n)) * 10.0 ** rng.integers(-8, 9, (n, n))
    x = rng.standard_normal(n)
    b = K @ x + rng.standard_normal(n) * 1e-9        # residuals far below the terms
    r = variants.exact_residual(K, x, b)
    for i in range(n):
        ex = Fraction(b[i]) - sum(Fraction(K[i, j]) * Fraction(x[j]) for j in range(n))
        assert r[i] == float(ex)


def test_refined_solve_reaches_the_exact_solution_where_lu_does_not():
    n = 9                                              # Hilbert matrix, condition ~5e11
    H = [[Fraction(1, i + j + 1) for j in range(n)] for i in range(n)]
    K = np.array([[float(v) for v in row] for row in H])
    xs = np.arange(1.0, n + 1.0)
    b = np.array([float(sum(Fraction(K[i, j]) * Fraction(xs[j]) for j in range(n))) for i in range(n)])
    # the exact solution of the FP64 system K x = b (rationals)
    M = [[Fraction(K[i, j]) for j in range(n)] + [Fraction(b[i])] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [M[r][k] - f * M[c][k] for k in range(n + 1)]
    exact = np.array([float(M[i][n] / M[i][i]) for i in range(n)])
    lu = np.linalg.solve(K, b)
    ref = variants.refined_solve(K, b)
    assert np.max(np.abs(lu - exact) / np.abs(exact)) > 1e-9
    assert np.max(np.abs(ref - exact) / np.abs(exact)) <= 4e-16


@pytest.mark.parametrize("i,j", [(-1, -1), (3, -1), (2, 11)])
def test_variants_agree_with_the_oracle_on_well_conditioned_scenarios(i, j):
    net = synth.make_network(14, 20, 5, 11, 1, seed=3, levels=(0.5,))
    ref = pipeline.evaluate(net, 0, i, j)
    outs = variants.outcomes(net, 0, i, j, processes=4)
    assert set(outs) == {"lu", "ldl", "refined"} | {f"perm{k}" for k in range(variants.N_PERM)}
    assert all(v == (int(ref["klass"]), int(ref["opf_iters"])) for v in outs.values())
    assert not variants.rounding_decided(outs)
    assert np.linalg.solve is not None and np.linalg.solve.__name__ == "solve"     # restored


def test_a_rounding_decided_118_bus_scenario():
    """Outage of branches 48 and 146 at 90 % load: the oracle's own LU reports no
    convergence in 50 iterations, the exactly refined steps converge in 41."""
    net = synth.case118()
    outs = variants.outcomes(net, 1, 48, 146, which=("lu", "refined"))
    assert outs["lu"] == (pipeline.OPF_NONCONV, 50)
    assert outs["refined"] == (pipeline.SECURE, 41)
    assert variants.rounding_decided(outs)


def test_permutation_alone_decides_a_118_bus_scenario():
    """Outage of branches 48 and 192 at 90 % load: LU of the system as formed converges
    in 44 iterations, LU of two symmetric permutations of the same systems never does."""
    net = synth.case118()
    outs = variants.outcomes(net, 1, 48, 192, which=("lu", "perm18", "perm22"), processes=3)
    assert outs == {"lu": (pipeline.SECURE, 44), "perm18": (pipeline.OPF_NONCONV, 50),
                    "perm22": (pipeline.OPF_NONCONV, 50)}
