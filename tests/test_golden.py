"""The stored expected values (tests/golden/*.json, written by make_golden.py from the
oracle alone) are still what the current oracle computes: a seeded sample of their
scenarios is re-evaluated here.  Classes and integers exactly; cost, max Re and min
damping ratio to 1e-9 relative (BLAS builds may round differently)."""
import importlib.util
import json
import os
import sys

import numpy as np
import pytest

from paper_2512_08465_gb300 import synth
from oracle import pipeline

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _make_golden():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_golden_files_come_from_the_current_oracle_sources():
    """The stored hash is that of the oracle modules (and input generator) the values
    come from: a change to any of them must be followed by make_golden.py."""
    h = _make_golden().oracle_hash()
    for name in ("case118_n1.json", "case118_pairs.json"):
        assert json.load(open(os.path.join(HERE, name)))["meta"]["oracle"] == h, name


@pytest.mark.parametrize("name,count", [("case118_n1.json", 5), ("case118_pairs.json", 4)])
def test_golden_sample_reproduces_from_the_oracle(name, count):
    gold = json.load(open(os.path.join(HERE, name)))
    assert gold["meta"]["network"] == "synth118" and gold["meta"]["damping_min"] == pipeline.DAMPING_MIN
    net = synth.case118()
    rows = gold["scenarios"]
    pick = np.random.default_rng(7).choice(len(rows), count, replace=False)
    for q in pick:
        g = rows[int(q)]
        r = pipeline.evaluate(net, g["level"], g["i"], g["j"])
        for k in ("klass", "severe", "n_islands", "opf_iters"):
            assert int(r[k]) == g[k], (name, q, k)
        for k in ("cost", "max_re", "min_zeta"):
            if g[k] is None:
                assert not np.isfinite(r[k]), (name, q, k)
            else:
                assert abs(r[k] - g[k]) <= 1e-9 * max(1.0, abs(g[k])), (name, q, k, r[k], g[k])
        if "Vm" in g:
            assert np.abs(np.asarray(r["Vm"]) - g["Vm"]).max() <= 1e-9



FULL = os.path.join(HERE, "case118_full.npz")


def test_full_study_tables_come_from_the_current_oracle():
    """The stored tables of the whole 118-bus study (make_full_golden.py) carry the
    hash of the current oracle sources, cover both levels completely, and a seeded
    sample of their scenarios re-evaluates to the stored values."""
    g = np.load(FULL)
    meta = json.loads(str(g["meta"]))
    assert meta["oracle"] == _make_golden().oracle_hash()
    net = synth.case118()
    E = net.n_elem
    n = 1 + E + E * (E - 1) // 2
    assert meta["scenarios_per_level"] == n
    for lv in (0, 1):
        k = g[f"{lv}_klass"]
        assert k.shape == (n,) and k.max() <= 6
        assert np.all((k == 1) == (g[f"{lv}_islands"] > 1))
    ii, jj = np.triu_indices(E, k=1)
    si = np.concatenate([[-1], np.arange(E), ii])
    sj = np.concatenate([[-1], -np.ones(E, np.int64), jj])
    rng = np.random.default_rng(31)
    for lv in (0, 1):
        for q in rng.choice(n, 3, replace=False):
            r = pipeline.evaluate(net, lv, int(si[q]), int(sj[q]))
            assert int(r["klass"]) == int(g[f"{lv}_klass"][q]) and int(r["opf_iters"]) == int(g[f"{lv}_iters"][q])
            for key, name in (("cost", "cost"), ("max_re", "max_re"), ("min_zeta", "min_zeta")):
                a, b = r[key], g[f"{lv}_{name}"][q]
                assert (np.isnan(a) and np.isnan(b)) or abs(a - b) <= 1e-9 * max(1.0, abs(b)), (lv, q, key)


def test_rounding_variant_table_comes_from_the_current_oracle():
    """tests/golden/case118_rounding_variants.json (make_rounding_variants.py): the
    current oracle's hash, every listed scenario, every variant, and -- on the kind of
    machine that wrote it -- two of its outcomes re-derived from the oracle."""
    import platform
    sys.path.insert(0, HERE)
    import make_rounding_variants as mrv
    from oracle import variants
    d = json.load(open(mrv.OUT))
    assert d["meta"]["oracle"] == _make_golden().oracle_hash()
    assert d["meta"]["variants"] == variants.names()
    assert [(e["level"], e["i"], e["j"]) for e in d["scenarios"]] == [tuple(s) for s in mrv.SCENARIOS]
    for e in d["scenarios"]:
        assert set(e["outcomes"]) == set(variants.names())
        assert len({tuple(v) for v in e["outcomes"].values()}) > 1      # each is rounding-decided
    if platform.machine() != d["meta"]["machine"]:
        pytest.skip("outcomes depend on the machine's floating-point library")
    e = next(e for e in d["scenarios"] if (e["level"], e["i"], e["j"]) == (1, 48, 192))
    outs = variants.outcomes(synth.case118(), 1, 48, 192, which=("lu", "perm18"), processes=2)
    assert outs == {k: tuple(e["outcomes"][k]) for k in ("lu", "perm18")}
