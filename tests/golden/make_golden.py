"""Write the stored expected values of the GPU parity tests.

Calls only the CPU oracle (``oracle/``) and the seeded input generator.  Run:
    python tests/golden/make_golden.py
Outputs (JSON text, committed):
  case118_n1.json     base + all 186 branch N-1 scenarios at the 70 % level
                      (the plain small configuration), classes and scalars for
                      all, bus voltages for the first 24 converged scenarios;
  case118_pairs.json  a seeded uniform sample of 150 unordered pairs of the 240
                      outage elements at each of the 70 % and 90 % levels.
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

import numpy as np  # noqa: E402

from paper_2512_08465_gb300 import synth  # noqa: E402
from oracle import pipeline  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
KEYS = ("level", "i", "j", "klass", "severe", "n_islands", "opf_iters", "converged", "cost", "max_re", "min_zeta")


# the oracle modules the stored values come from, and the input generator
SOURCES = ("oracle/grid.py", "oracle/opf.py", "oracle/dynamics.py", "oracle/eig.py", "oracle/eig.c",
           "oracle/pipeline.py", "paper_2512_08465_gb300/synth.py")


def oracle_hash():
    h = hashlib.sha256()
    for rel in SOURCES:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:16]


def _clean(r, volt):
    d = {k: (None if isinstance(r[k], float) and not np.isfinite(r[k]) else
             (int(r[k]) if isinstance(r[k], (bool, np.bool_, np.integer)) else r[k])) for k in KEYS}
    for k in ("cost", "max_re", "min_zeta"):
        if d[k] is not None:
            d[k] = float(d[k])
    if volt and "Vm" in r:
        d["Vm"] = [float(v) for v in r["Vm"]]
        d["Va"] = [float(v) for v in r["Va"]]
    return d


def pair_sample(E, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    ks = np.sort(rng.choice(E * (E - 1) // 2, size=n, replace=False))
    ii, jj = np.triu_indices(E, k=1)
    return [(int(ii[k]), int(jj[k])) for k in ks]


def main():
    net = synth.case118()
    procs = os.cpu_count() or 1
    sc = [(0, -1, -1)] + [(0, e, -1) for e in range(net.n_branch)]
    res = pipeline.evaluate_many(net, sc, procs)
    nv = 0
    rows = []
    for r in res:
        volt = r.get("converged") and nv < 24
        nv += bool(volt)
        rows.append(_clean(r, volt))
    meta = dict(network="synth118", seed=net.seed, levels=list(net.levels), oracle=oracle_hash(),
                damping_min=pipeline.DAMPING_MIN)
    json.dump(dict(meta=meta, scenarios=rows), open(os.path.join(HERE, "case118_n1.json"), "w"))
    pairs = pair_sample(net.n_elem, 150, 2512)
    sc = [(lv, i, j) for lv in (0, 1) for (i, j) in pairs]
    res = pipeline.evaluate_many(net, sc, procs)
    rows = [_clean(r, False) for r in res]
    json.dump(dict(meta=meta, scenarios=rows), open(os.path.join(HERE, "case118_pairs.json"), "w"))


if __name__ == "__main__":
    main()
