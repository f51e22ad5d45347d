"""Serving path: continuous batching across requests and networks, admission
by device-memory footprint (cs_submit_contingencies / cs_poll).

Each scenario is evaluated by its own CTA, independently of what else is in
its launch, so a request's records must equal, bit for bit, those of the same
scenarios evaluated directly with cs_evaluate_device.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2512_08465_gb300 import cs, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
FIELDS = ("klass", "severe", "n_islands", "opf_iters", "cost", "max_re", "min_zeta",
          "v_margin", "max_loading", "shed_mw", "main_klass")


@pytest.fixture(scope="module")
def nets():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    small = synth.make_network(14, 20, 5, 11, 1, seed=3, levels=(0.5, 0.8))
    return small, synth.case118()


def _direct(ctx, nid, level, ei, ej):
    ti = torch.as_tensor(np.asarray(ei, np.int32), device=DEV)
    tj = torch.as_tensor(np.asarray(ej, np.int32), device=DEV)
    out = ctx.alloc_results(ti.numel(), DEV, indices=True, main_island=True)
    ctx.evaluate_device(nid, level, ti, tj, out)
    ctx.sync()
    return {k: out[k].cpu().numpy() for k in FIELDS}


def _requests(rng, net, n_req, lo=1, hi=200):
    ii, jj = synth.all_pairs(net.n_elem)
    reqs = []
    for _ in range(n_req):
        m = int(rng.integers(lo, hi + 1))
        sel = rng.choice(ii.size, m, replace=False)
        reqs.append((ii[sel].astype(np.int32), jj[sel].astype(np.int32)))
    return reqs


def test_batched_requests_across_networks_equal_direct_evaluation(nets):
    small, big = nets
    ctx = cs.Context(precision=cs.PREC_MIXED)
    ids = {0: ctx.load_network(small), 1: ctx.load_network(big)}
    rng = np.random.default_rng(11)
    work = []
    for which, net in ((0, small), (1, big)):
        for level in (0, 1):
            for ei, ej in _requests(rng, net, 12, hi=60 if which == 0 else 150):
                work.append((which, level, ei, ej))
    order = rng.permutation(len(work))
    rids = [(work[q], ctx.submit(ids[work[q][0]], work[q][1], work[q][2], work[q][3])) for q in order]
    got = [(w, ctx.poll(r, 600_000_000)) for w, r in rids]
    stats = ctx.serving_stats()
    assert stats["completed"] == len(work) and stats["queued"] == 0 and stats["in_flight"] == 0
    assert stats["batches"] < len(work)           # queued requests of one (network, level) were merged
    assert stats["merged"] == len(work) - stats["batches"]
    ref_ctx = cs.Context(precision=cs.PREC_MIXED)
    ref_ids = {0: ref_ctx.load_network(small), 1: ref_ctx.load_network(big)}
    for (which, level, ei, ej), out in got:
        ref = _direct(ref_ctx, ref_ids[which], level, ei, ej)
        for k in FIELDS:
            np.testing.assert_array_equal(out[k], ref[k], err_msg=k)
    ref_ctx.close()
    ctx.close()


def test_poll_pending_then_done_and_empty_request(nets):
    small, big = nets
    ctx = cs.Context(precision=cs.PREC_MIXED)
    nid = ctx.load_network(big)
    ii, jj = synth.all_pairs(big.n_elem)
    rid = ctx.submit(nid, 1, ii[:4096], jj[:4096])
    assert ctx.poll(rid, 0) is None               # a 4096-pair request takes far longer than a poll
    out = ctx.poll(rid, 600_000_000)
    assert out is not None and out["klass"].shape == (4096,)
    e = ctx.submit(nid, 0, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert ctx.poll(e, 0) is not None
    with pytest.raises(cs.CSError):
        ctx.poll(rid, 0)                          # released by the successful poll
    ctx.close()


def test_hbm_budget_admission(nets):
    small, big = nets
    tiny = cs.Context(precision=cs.PREC_MIXED, hbm_budget=1 << 16)
    with pytest.raises(cs.CSError) as ei:
        tiny.load_network(big)                    # 118-bus tables alone exceed 64 KB
    assert ei.value.status == cs.CS_E_NOMEM
    tiny.close()
    # a budget that holds the network and a small workspace: batches shrink their chunk
    probe = cs.Context(precision=cs.PREC_MIXED)
    pid = probe.load_network(big)
    held = probe.serving_stats()["bytes_now"]
    probe.close()
    budget = held + (2 << 30)
    ctx = cs.Context(precision=cs.PREC_MIXED, hbm_budget=budget, serve_slots=2)
    nid = ctx.load_network(big)
    ii, jj = synth.all_pairs(big.n_elem)
    rng = np.random.default_rng(4)
    sel = rng.choice(ii.size, 3000, replace=False)
    rids = [ctx.submit(nid, 0, ii[sel[q:q + 1000]], jj[sel[q:q + 1000]]) for q in range(0, 3000, 1000)]
    outs = [ctx.poll(r, 600_000_000) for r in rids]
    st = ctx.serving_stats()
    assert st["peak_bytes"] <= budget and st["nomem"] == 0 and st["completed"] == 3
    ref = cs.Context(precision=cs.PREC_MIXED)
    rid_ = ref.load_network(big)
    want = _direct(ref, rid_, 0, ii[sel], jj[sel])
    got = {k: np.concatenate([o[k] for o in outs]) for k in FIELDS}
    for k in FIELDS:
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    ref.close()
    ctx.close()


def test_main_island_requests_equal_direct_evaluation(nets):
    """With the main-island form on, requests of islanded and connected pairs return the
    main-island fields (shed, class of the main island, its OPF cost and indices) equal,
    bit for bit, to direct evaluation."""
    from oracle import grid
    small, big = nets
    ii, jj = synth.all_pairs(big.n_elem)
    rng = np.random.default_rng(31)
    sel = rng.choice(ii.size, 1500, replace=False)
    isl = np.array([grid.count_islands(big.n_bus, *(lambda sc: (big.f[sc.br], big.t[sc.br]))(
        grid.make_scenario(big, 0, int(ii[q]), int(jj[q])))) > 1 for q in sel])
    assert isl.sum() > 50
    ctx = cs.Context(precision=cs.PREC_MIXED, main_island=1)
    nid = ctx.load_network(big)
    rids = [ctx.submit(nid, 1, ii[sel[q:q + 500]], jj[sel[q:q + 500]]) for q in range(0, 1500, 500)]
    outs = [ctx.poll(r, 600_000_000) for r in rids]
    got = {k: np.concatenate([o[k] for o in outs]) for k in FIELDS}
    want = _direct(ctx, nid, 1, ii[sel], jj[sel])
    for k in FIELDS:
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    assert np.all(got["main_klass"][isl] != 255) and np.all(got["main_klass"][~isl] == 255)
    assert np.all(got["shed_mw"][~isl] == 0.0) and np.all(got["shed_mw"][isl] >= 0.0)
    ctx.close()


def test_requests_split_over_batches_equal_direct_evaluation(nets):
    """With a batch cap below the request sizes every request is split over several
    batches (and slots); each request still completes with all its records, equal bit
    for bit to direct evaluation, and small requests submitted after a large one are
    served without waiting for all of it."""
    small, big = nets
    ctx = cs.Context(precision=cs.PREC_MIXED, batch_cap=96, serve_slots=3)
    nid = ctx.load_network(big)
    rng = np.random.default_rng(19)
    reqs = _requests(rng, big, 6, lo=150, hi=400) + _requests(rng, big, 4, lo=5, hi=40)
    rids = [ctx.submit(nid, 1, ei, ej) for ei, ej in reqs]
    for (ei, ej), rid in zip(reqs, rids):
        got = ctx.poll(rid, 600_000_000)
        ref = _direct(ctx, nid, 1, ei, ej)
        for k in FIELDS:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    st = ctx.serving_stats()
    total = sum(ei.size for ei, _ in reqs)
    assert st["completed"] == len(reqs) and st["batches"] >= total // 96
    ctx.close()
