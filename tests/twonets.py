"""Two networks built apart and joined by one tie branch, by a construction of the
tests' own (shared by the main-island tests on CPU and GPU)."""
import copy

import numpy as np

from paper_2512_08465_gb300 import synth


def pair():
    """The two networks: 14 buses / 5 units and 9 buses / 3 units, 50 % load."""
    A = synth.make_network(14, 20, 5, 11, 1, seed=3, levels=(0.5,))
    Bn = synth.make_network(9, 12, 3, 6, 0, seed=5, levels=(0.5,))
    return A, Bn


def join(A, Bn, a_bus, b_bus, ref):
    """A and B side by side (B's buses after A's), plus one tie branch a_bus - (nA + b_bus),
    the last branch; ref is the joined network's reference bus."""
    nA = A.n_bus
    J = copy.copy(A)
    for k in ("Vmin", "Vmax", "Gs", "Bs", "Pd_shape", "Qd_shape"):
        setattr(J, k, np.concatenate([getattr(A, k), getattr(Bn, k)]))
    J.Pd = np.concatenate([A.Pd, Bn.Pd], axis=1)
    J.Qd = np.concatenate([A.Qd, Bn.Qd], axis=1)
    J.f = np.concatenate([A.f, Bn.f + nA, [a_bus]]).astype(np.int32)
    J.t = np.concatenate([A.t, Bn.t + nA, [nA + b_bus]]).astype(np.int32)
    tie = dict(r=0.01, x=0.05, b=0.0, rate=300.0, tap=1.0, kind=synth.KIND_LINE)
    for k, v in tie.items():
        J.__dict__[k] = np.concatenate([getattr(A, k), getattr(Bn, k), [v]]).astype(getattr(A, k).dtype)
    J.gbus = np.concatenate([A.gbus, Bn.gbus + nA]).astype(np.int32)
    for k in ("Pmin", "Pmax", "Qmin", "Qmax", "c2", "c1", "c0", "H", "D",
              "xd", "xq", "xdp", "Td0p", "Tq0p", "KA", "TA"):
        setattr(J, k, np.concatenate([getattr(A, k), getattr(Bn, k)]))
    J.ref_bus = int(ref)
    return J
