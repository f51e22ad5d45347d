"""N-3 extension and common-cause pair frequencies (the paper's outlook) on the
GPU against the CPU oracle: triple enumeration, N-3 scenario parity, and the
Risk Index with explicit pair frequencies (exact, so compared bit for bit)."""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2512_08465_gb300 import cs, synth  # noqa: E402
from oracle import pipeline, risk  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    net = synth.make_network(14, 20, 5, 11, 1, seed=3, levels=(0.5,))
    c = cs.Context(precision=cs.PREC_MIXED)
    nid = c.load_network(net)
    yield net, c, nid
    c.close()


def _t(a):
    return torch.as_tensor(np.asarray(a, np.int32), device=DEV)


def test_enumerate_triples_matches_itertools():
    E = 25
    ref = np.array(list(itertools.combinations(range(E), 3)), np.int32)
    ei, ej, ek = (torch.empty(ref.shape[0], dtype=torch.int32, device=DEV) for _ in range(3))
    cs.enumerate_triples_device(E, 0, ref.shape[0], ei, ej, ek)
    np.testing.assert_array_equal(np.stack([ei.cpu().numpy(), ej.cpu().numpy(), ek.cpu().numpy()], 1), ref)
    part = [torch.empty(100, dtype=torch.int32, device=DEV) for _ in range(3)]
    cs.enumerate_triples_device(E, 1000, 100, *part)
    np.testing.assert_array_equal(np.stack([p.cpu().numpy() for p in part], 1), ref[1000:1100])
    with pytest.raises(cs.CSError):
        cs.enumerate_triples_device(E, ref.shape[0] - 5, 10, *part)


def test_n3_scenarios_match_oracle(setup):
    net, c, nid = setup
    E = net.n_elem
    rng = np.random.default_rng(31)
    trip = np.array(list(itertools.combinations(range(E), 3)))
    sel = trip[rng.choice(len(trip), 24, replace=False)]
    out = c.alloc_results(len(sel), DEV)
    c.evaluate_device_n3(nid, 0, _t(sel[:, 0]), _t(sel[:, 1]), _t(sel[:, 2]), out)
    c.sync()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    for q, (i, j, k) in enumerate(sel):
        ref = pipeline.evaluate(net, 0, int(i), int(j), k=int(k))
        assert int(got["klass"][q]) == ref["klass"], (i, j, k, got["klass"][q], ref["klass"])
        assert int(got["n_islands"][q]) == ref["n_islands"]
        if ref["converged"]:
            assert abs(got["cost"][q] - ref["cost"]) <= 1e-6 * abs(ref["cost"])
        if ref["converged"]:
            assert int(got["opf_iters"][q]) == ref["opf_iters"], (i, j, k)
        if np.isfinite(ref["max_re"]):                # mixed form: refined in FP64
            assert abs(got["max_re"][q] - ref["max_re"]) <= 1e-6
            assert abs(got["min_zeta"][q] - ref["min_zeta"]) <= 1e-6
    # a missing third element is the N-2 evaluation, record for record
    ii, jj = sel[:, 0], sel[:, 1]
    a = c.alloc_results(len(sel), DEV)
    b = c.alloc_results(len(sel), DEV)
    c.evaluate_device(nid, 0, _t(ii), _t(jj), a)
    c.evaluate_device_n3(nid, 0, _t(ii), _t(jj), _t(-np.ones(len(sel))), b)
    c.sync()
    for k in ("klass", "cost", "max_re", "min_zeta", "opf_iters"):
        np.testing.assert_array_equal(a[k].cpu().numpy(), b[k].cpu().numpy())


def test_risk_index_pair_freq_matches_oracle(setup):
    net, c, nid = setup
    E = net.n_elem
    ii, jj = synth.all_pairs(E)
    out = c.alloc_results(E + ii.size, DEV)
    c.evaluate_device(nid, 0, _t(np.concatenate([np.arange(E), ii])), _t(np.concatenate([-np.ones(E), jj])), out)
    c.sync()
    sev = out["severe"].cpu().numpy()
    S1 = sev[:E]
    S2 = np.zeros((E, E), np.uint8)
    S2[ii, jj] = sev[E:]
    S2 = S2 + S2.T
    lam = synth.failure_rates(E, 41)
    rng = np.random.default_rng(42)
    F = rng.uniform(1e-4, 0.2, (E, E))
    F = 0.5 * (F + F.T)
    for mode in (cs.RISK_EQ3, cs.RISK_ORDERED):
        om = risk.ORDERED if mode else risk.EQ3
        R, missing = c.risk_index_pair_freq(nid, 0, lam, F, mode)
        assert missing == 0
        np.testing.assert_array_equal(R, risk.risk_index_pair_freq(lam, F, S1, S2, om))
        Rp, _ = c.risk_index_pair_freq(nid, 0, lam, np.outer(lam, lam), mode)
        Rs, _ = c.risk_index(nid, 0, lam, mode)
        np.testing.assert_array_equal(Rp, Rs)
    with pytest.raises(cs.CSError):
        c.risk_index_pair_freq(nid, 0, lam, -F, cs.RISK_EQ3)
