"""Oracle Risk Index against the worked values of Section V and brute force."""
import math

import numpy as np

from oracle import risk


def _table_i(n_line=175, n_tr=11, n_gen=53):
    return np.array([0.05] * n_line + [0.02] * n_tr + [0.10] * n_gen)


def test_printed_values_all_severe_ordered():
    """Section V: a line whose every scenario is severe has R = 1.472 and the
    transformers lie between 0.56 and 0.59; both need the ordered reading."""
    lam = _table_i()
    E = lam.size
    R = risk.risk_index(lam, np.ones(E), np.ones((E, E)), risk.ORDERED)
    assert abs(R[0] - 1.472) < 1e-12
    assert abs(R[175] - 0.590) < 1e-12
    assert abs(R[186] - 2.934) < 1e-12


def test_literal_eq3_values():
    lam = _table_i()
    E = lam.size
    R = risk.risk_index(lam, np.ones(E), np.ones((E, E)), risk.EQ3)
    assert abs(R[0] - 0.761) < 1e-12
    assert abs(R[175] - 0.305) < 1e-12


def test_exact_against_fsum_and_brute_force_lists():
    rng = np.random.default_rng(8)
    E = 30
    lam = rng.uniform(0.01, 1.0, E)
    S1 = rng.integers(0, 2, E)
    U = np.triu(rng.integers(0, 2, (E, E)), 1)
    S2 = U + U.T
    for mode, mult in ((risk.EQ3, 1), (risk.ORDERED, 2)):
        R = risk.risk_index(lam, S1, S2, mode)
        for i in range(E):
            terms = [lam[i]] if S1[i] else []
            for j in range(E):
                if j != i and S2[i, j]:
                    terms += [lam[i] * lam[j]] * mult
            assert R[i] == math.fsum(terms)         # fsum is correctly rounded
    unordered = [(i, j, S2[i, j]) for i in range(E) for j in range(i + 1, E)]
    ordered = [(i, j, S2[i, j]) for i in range(E) for j in range(E) if i != j]
    np.testing.assert_array_equal(risk.risk_index(lam, S1, S2, risk.EQ3),
                                  risk.risk_index_ordered_list(lam, S1, unordered))
    np.testing.assert_array_equal(risk.risk_index(lam, S1, S2, risk.ORDERED),
                                  risk.risk_index_ordered_list(lam, S1, ordered))


def test_zero_severity_gives_zero():
    lam = np.full(5, 0.3)
    np.testing.assert_array_equal(risk.risk_index(lam, np.zeros(5), np.zeros((5, 5))), 0.0)


def test_pair_frequency_form_reduces_to_eq3_and_matches_brute_force():
    """Explicit pair frequencies (common-cause extension): with F_ij = fl(l_i l_j)
    it is Eq. 3 exactly; for a general F it is the exact rational sum, rounded once."""
    from fractions import Fraction
    import numpy as np
    from oracle import risk
    rng = np.random.default_rng(9)
    E = 11
    lam = rng.uniform(0.01, 1.0, E)
    S1 = rng.integers(0, 2, E)
    S2 = np.triu(rng.integers(0, 2, (E, E)), 1)
    S2 = S2 + S2.T
    Fprod = np.outer(lam, lam)                        # fl(l_i l_j) elementwise
    for mode in (risk.EQ3, risk.ORDERED):
        np.testing.assert_array_equal(risk.risk_index_pair_freq(lam, Fprod, S1, S2, mode),
                                      risk.risk_index(lam, S1, S2, mode))
    F = rng.uniform(1e-4, 0.3, (E, E))                # e.g. a common-cause model, not a product
    F = 0.5 * (F + F.T)
    got = risk.risk_index_pair_freq(lam, F, S1, S2, risk.EQ3)
    for i in range(E):
        want = (Fraction(lam[i]) if S1[i] else Fraction(0)) + sum(
            (Fraction(F[i, j]) for j in range(E) if j != i and S2[i, j]), Fraction(0))
        assert got[i] == float(want)
    got2 = risk.risk_index_pair_freq(lam, F, S1, S2, risk.ORDERED)
    for i in range(E):                                # ordered = Eq. 3 pair term counted twice, exactly
        want = (Fraction(lam[i]) if S1[i] else Fraction(0)) + 2 * sum(
            (Fraction(F[i, j]) for j in range(E) if j != i and S2[i, j]), Fraction(0))
        assert got2[i] == float(want)
