"""Writes tests/golden/case118_rounding_variants.json: for each listed scenario of
the 118-bus study, the oracle pipeline's outcome (class, interior-point iterations)
under every rounding-level variant of its Newton-step solve (oracle/variants.py).

Only the oracle runs here.  The scenarios listed are those whose OPF outcome has
differed between the GPU and the stored oracle tables in some build, so they get
this extra analysis; which outcomes each variant gives is the oracle's alone.
FP64 rounding, including that of the machine's BLAS, decides these scenarios: the
same variants give other outcomes on another CPU, so the stored table records the
machine it was made on and the test takes the union of stored and live outcomes.

    python tests/golden/make_rounding_variants.py [processes]
"""
import json
import os
import platform
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

SCENARIOS = [(1, 14, 112), (1, 23, 112), (1, 39, 112), (1, 112, 171), (1, 48, 146), (1, 48, 192),
             (1, 179, 232), (1, 48, 80), (1, 48, 165), (1, 48, 198), (1, 48, 205), (1, 48, 223),
             (1, 187, 232)]
OUT = os.path.join(HERE, "case118_rounding_variants.json")


def main():
    from paper_2512_08465_gb300 import synth
    from oracle import variants
    import make_golden
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    net = synth.case118()
    table = []
    for lv, i, j in SCENARIOS:
        outs = variants.outcomes(net, lv, i, j, processes=procs)
        table.append({"level": lv, "i": i, "j": j, "outcomes": {k: list(v) for k, v in outs.items()}})
        print((lv, i, j), sorted(set(outs.values())), flush=True)
    meta = {"network": "synth118", "oracle": make_golden.oracle_hash(), "machine": platform.machine(),
            "variants": variants.names()}
    with open(OUT, "w") as f:
        json.dump({"meta": meta, "scenarios": table}, f, indent=1)


if __name__ == "__main__":
    main()
