"""cs_risk_index_static (static device scratch, no allocation) against
cs_risk_index on the same severity table.

The reduction is exact (fixed point, one rounding), so the tolerance is zero:
both entry points must return the same doubles and the same missing-pair
count.  The file is collected last on purpose, so that the static entry point
also runs after every other GPU test in the session has used the device.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2512_08465_gb300 import cs, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cs.Context()
    yield c
    c.close()


def _evaluate(ctx, nid, level, ei, ej):
    dev = torch.device("cuda:0")
    ei = torch.as_tensor(np.asarray(ei, np.int32), device=dev)
    ej = torch.as_tensor(np.asarray(ej, np.int32), device=dev)
    out = ctx.alloc_results(ei.numel(), dev)
    ctx.evaluate_device(nid, level, ei, ej, out)
    ctx.sync()


def test_static_risk_index_equals_allocating_entry_point(ctx):
    net = synth.make_network(14, 20, 5, 11, 1, seed=3, levels=(0.5, 0.9))
    nid = ctx.load_network(net)
    E = net.n_elem
    ii, jj = synth.all_pairs(E)
    # level 0: every N-1 and every pair; level 1: N-1 and every third pair
    _evaluate(ctx, nid, 0, np.concatenate([np.arange(E), ii]), np.concatenate([-np.ones(E), jj]))
    sel = np.arange(0, ii.size, 3)
    _evaluate(ctx, nid, 1, np.concatenate([np.arange(E), ii[sel]]), np.concatenate([-np.ones(E), jj[sel]]))
    for call, seed in enumerate((11, 12)):          # two calls in a row, different rates
        lam = synth.failure_rates(E, seed)
        for level, missing in ((0, 0), (1, ii.size - sel.size)):
            for mode in (cs.RISK_EQ3, cs.RISK_ORDERED):
                R_ref, m_ref = ctx.risk_index(nid, level, lam, mode)
                R_st, m_st = ctx.risk_index_static(nid, level, lam, mode)
                assert m_ref == missing and m_st == missing, (call, level, mode)
                np.testing.assert_array_equal(R_st, R_ref)
                assert np.all(R_st >= 0.0)
    ctx.unload_network(nid)


def test_static_risk_index_validates_like_the_allocating_one(ctx):
    net = synth.make_network(14, 20, 5, 11, 1, seed=3, levels=(0.5,))
    nid = ctx.load_network(net)
    lam = synth.failure_rates(net.n_elem, 1)
    with pytest.raises(cs.CSError):
        ctx.risk_index_static(nid, 1, lam)                    # no such level
    bad = lam.copy()
    bad[0] = 0.0
    with pytest.raises(cs.CSError):
        ctx.risk_index_static(nid, 0, bad)                    # lambda outside [2^-30, 2^10]
    with pytest.raises(cs.CSError):
        ctx.risk_index_static(nid + 1000, 0, lam)             # unknown network
    ctx.unload_network(nid)


def _replicated(net, k):
    """The same electrical network with every branch split into k identical parallel
    branches (impedance x k, charging and rating / k), so that it has k times the
    branch outage elements."""
    import dataclasses
    rep = lambda a: np.repeat(a, k)
    return dataclasses.replace(net, f=rep(net.f), t=rep(net.t), r=rep(net.r) * k, x=rep(net.x) * k,
                               b=rep(net.b) / k, rate=rep(net.rate) / k, tap=rep(net.tap), kind=rep(net.kind))


def test_static_risk_index_rejects_networks_beyond_its_scratch(ctx):
    """More than 4096 outage elements do not fit the static scratch: CS_E_ARG with a
    message naming the limit, while the allocating entry point still answers."""
    base = synth.make_network(14, 20, 5, 11, 1, seed=3, levels=(0.5,))
    net = _replicated(base, 205)                          # 4100 branches + 5 generators
    assert net.n_elem == 4105
    nid = ctx.load_network(net)
    lam = synth.failure_rates(net.n_elem, 3)
    with pytest.raises(cs.CSError) as err:
        ctx.risk_index_static(nid, 0, lam)
    assert "4096" in str(err.value)
    R, missing = ctx.risk_index(nid, 0, lam)
    assert R.shape == (net.n_elem,) and missing == net.n_elem * (net.n_elem + 1) // 2
    assert np.all(R == 0.0)                                # nothing evaluated yet
    ctx.unload_network(nid)
