"""Risk Index R_i, computed exactly (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section II-C: F_i = lambda_i (Eq. 1), F_ij = lambda_i lambda_j (Eq. 2) and
R_i = F_i S_i + sum_{j != i} F_ij S_ij (Eq. 3).

Exactness.  Each pair frequency is the IEEE double product fl(lambda_i lambda_j);
the sum of the N-1 term and all pair terms is carried out exactly with Python
rationals and rounded once to the nearest double (ties to even).  The result is
therefore independent of summation order, so any implementation that rounds the
same exact value must agree bit for bit.

Two readings of the pair sum (the paper is inconsistent here):

* ``EQ3``     each unordered pair {i, j} contributes once, as Eq. 3 is written;
* ``ORDERED`` both orderings (i, j) and (j, i) of the ordered N-2 enumeration of
  Section II-A contribute, i.e. the pair sum counts twice.  This reproduces the
  values printed in Section V (a line with every scenario severe under the
  Table I rates gives R = 1.472, a transformer 0.590).

Pinned in ``tests/test_oracle_risk.py`` by those printed values, by the literal
Eq. 3 values (0.761, 0.305) and by brute force over explicit ordered scenario
lists.
"""
from __future__ import annotations

from fractions import Fraction
import numpy as np

EQ3 = 0
ORDERED = 1


def risk_index(lam, S1, S2, mode: int = ORDERED):
    """R for every element.

    lam : failure rates, length E (per year)
    S1  : N-1 severities, length E (0/1)
    S2  : E x E symmetric 0/1 matrix of unordered-pair severities (diagonal ignored)
    """
    lam = [float(v) for v in lam]
    E = len(lam)
    S2 = np.asarray(S2)
    mult = 2 if mode == ORDERED else 1
    out = np.zeros(E)
    for i in range(E):
        acc = Fraction(lam[i]) if int(S1[i]) else Fraction(0)
        pair = Fraction(0)
        for j in range(E):
            if j != i and int(S2[i, j]):
                pair += Fraction(lam[i] * lam[j])
        out[i] = float(acc + mult * pair)
    return out


def risk_index_pair_freq(lam, F, S1, S2, mode: int = ORDERED):
    """R with explicit pair frequencies: R_i = lambda_i S_i + m sum_{j != i} F_ij S_ij.

    The extension to common-cause pair frequencies named in the paper's outlook
    (Section VI): F_ij (per year, row i used for element i) replaces the
    independent-failure product of Eq. 2.  Exact over the given doubles, rounded
    once; with F_ij = fl(lambda_i lambda_j) it is ``risk_index``."""
    lam = [float(v) for v in lam]
    E = len(lam)
    F = np.asarray(F, dtype=np.float64)
    S2 = np.asarray(S2)
    mult = 2 if mode == ORDERED else 1
    out = np.zeros(E)
    for i in range(E):
        acc = Fraction(lam[i]) if int(S1[i]) else Fraction(0)
        pair = Fraction(0)
        for j in range(E):
            if j != i and int(S2[i, j]):
                pair += Fraction(float(F[i, j]))
        out[i] = float(acc + mult * pair)
    return out


def risk_index_ordered_list(lam, S1, ordered_pairs):
    """Brute-force form: Eq. 3 summed over an explicit list of ordered N-2
    scenarios (i, j, S_ij) in which i is the first outage; the pair frequency
    F_ij of a scenario is charged to both elements it involves."""
    lam = [float(v) for v in lam]
    E = len(lam)
    acc = [Fraction(lam[i]) if int(S1[i]) else Fraction(0) for i in range(E)]
    for (i, j, s) in ordered_pairs:
        if int(s):
            acc[i] += Fraction(lam[i] * lam[j])
            acc[j] += Fraction(lam[i] * lam[j])
    return np.array([float(a) for a in acc])
