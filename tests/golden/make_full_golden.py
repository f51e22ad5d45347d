"""Write the oracle's severity tables of the whole 118-bus N-2 study.

Calls only the CPU oracle (``oracle/``) and the seeded input generator.  The
workload is the full enumeration of Section II-A on the seeded 118-bus network:
at each of the two load levels (70 %, 90 %) the base case, the 240 single
outages (186 branches, 54 generators) and all 28,680 unordered pairs of the 240
outage elements -- 57,842 scenarios.  Run (about 1.5 h on 8 cores):
    python tests/golden/make_full_golden.py [processes]
Output (committed): ``case118_full.npz`` with, per level L in {0, 1},
  L_klass    uint8[28,921]   class of base, N-1 (element order), pairs (i < j,
                             row-major over i as numpy.triu_indices)
  L_islands  int16, L_iters int16, L_cost / L_max_re / L_min_zeta float64
and ``meta`` (JSON text): network, seed, oracle hash, damping threshold.
Progress is kept in ``case118_full.partial.npz`` so an interrupted run resumes.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

import numpy as np  # noqa: E402

from paper_2512_08465_gb300 import synth  # noqa: E402
from oracle import pipeline  # noqa: E402
from make_golden import oracle_hash  # noqa: E402

OUT = os.path.join(HERE, "case118_full.npz")
PART = os.path.join(HERE, "case118_full.partial.npz")
FIELDS = (("klass", np.uint8), ("islands", np.int16), ("iters", np.int16),
          ("cost", np.float64), ("max_re", np.float64), ("min_zeta", np.float64))


def scenarios(E):
    """(i, j) of one level in stored order: base, N-1, then the pairs."""
    ii, jj = np.triu_indices(E, k=1)
    i = np.concatenate([[-1], np.arange(E), ii]).astype(np.int64)
    j = np.concatenate([[-1], -np.ones(E, np.int64), jj]).astype(np.int64)
    return i, j


def main():
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    net = synth.case118()
    E = net.n_elem
    si, sj = scenarios(E)
    n = si.size
    h = oracle_hash()
    tab = {f"{lv}_{k}": np.zeros(n, t) for lv in (0, 1) for k, t in FIELDS}
    done = {lv: 0 for lv in (0, 1)}
    if os.path.exists(PART):
        p = np.load(PART)
        if str(p["hash"]) == h:
            for k in tab:
                tab[k][:] = p[k]
            done = {0: int(p["done0"]), 1: int(p["done1"])}
    chunk = 2048
    t0 = time.time()
    for lv in (0, 1):
        while done[lv] < n:
            a, b = done[lv], min(n, done[lv] + chunk)
            res = pipeline.evaluate_many(net, [(lv, int(si[q]), int(sj[q])) for q in range(a, b)], procs)
            for q, r in zip(range(a, b), res):
                assert r["i"] == si[q] and r["j"] == sj[q] and r["level"] == lv
                tab[f"{lv}_klass"][q] = r["klass"]
                tab[f"{lv}_islands"][q] = r["n_islands"]
                tab[f"{lv}_iters"][q] = r["opf_iters"]
                tab[f"{lv}_cost"][q] = r["cost"]
                tab[f"{lv}_max_re"][q] = r["max_re"]
                tab[f"{lv}_min_zeta"][q] = r["min_zeta"]
            done[lv] = b
            np.savez(PART, hash=h, done0=done[0], done1=done[1], **tab)
            print(f"level {lv}: {b}/{n}  {time.time() - t0:.0f} s", flush=True)
    meta = dict(network="synth118", seed=net.seed, levels=list(net.levels), oracle=h,
                damping_min=pipeline.DAMPING_MIN, elements=E, scenarios_per_level=n)
    np.savez_compressed(OUT, meta=json.dumps(meta), **tab)
    os.remove(PART)


if __name__ == "__main__":
    main()
