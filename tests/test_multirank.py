"""Multi-rank host logic on CPU (gloo, world size 2): contiguous pair blocks,
the max-over-ranks step time, and the severity merge of a sharded network,
whose Risk Index must equal the single-rank one bit for bit.  The severities
come from the CPU oracle on a small seeded network."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2512_08465_gb300 import shard, synth  # noqa: E402


def _net():
    return synth.make_network(9, 12, 3, 6, 0, seed=5, levels=(0.5,))


def _worker(rank, world, port, outq):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OPENBLAS_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import pipeline
    net = _net()
    E = net.n_elem
    ii, jj = synth.all_pairs(E)
    first, count = shard.pair_block(rank, world, ii.size)
    tab = np.full(ii.size, shard.MISSING, np.uint8)
    for k in range(first, first + count):
        tab[k] = pipeline.evaluate(net, 0, int(ii[k]), int(jj[k]))["severe"]
    merged = shard.merge_severity(tab)
    # the in-place tensor form the benchmark uses on device tables (here a CPU tensor)
    flat = torch.from_numpy(tab.copy())
    shard.merge_severity_device(flat)
    step = shard.max_over_ranks(1.5 + rank)
    if rank == 0:
        outq.put((merged, step, flat.numpy().copy()))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_pair_blocks_cover_exactly_once():
    for total in (0, 1, 7, 28680):
        for world in (1, 2, 3, 8):
            spans = [shard.pair_block(r, world, total) for r in range(world)]
            assert spans[0][0] == 0 and sum(c for _, c in spans) == total
            for (f0, c0), (f1, _) in zip(spans, spans[1:]):
                assert f0 + c0 == f1
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1


def test_two_ranks_merge_equals_single_rank():
    from oracle import pipeline, risk
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged, step, merged_t = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert step == 2.5                                  # max over ranks of 1.5 + rank
    net = _net()
    E = net.n_elem
    ii, jj = synth.all_pairs(E)
    single = np.array([pipeline.evaluate(net, 0, int(a), int(b))["severe"] for a, b in zip(ii, jj)], np.uint8)
    np.testing.assert_array_equal(merged, single)        # every pair evaluated by exactly one rank
    np.testing.assert_array_equal(merged_t, single)      # the in-place tensor merge agrees
    S1 = np.array([pipeline.evaluate(net, 0, i, -1)["severe"] for i in range(E)], np.uint8)
    S2 = np.zeros((E, E), np.uint8)
    S2[ii, jj] = merged
    S2 = S2 + S2.T
    S2s = np.zeros((E, E), np.uint8)
    S2s[ii, jj] = single
    S2s = S2s + S2s.T
    lam = synth.failure_rates(E, 3)
    for mode in (risk.EQ3, risk.ORDERED):
        np.testing.assert_array_equal(risk.risk_index(lam, S1, S2, mode), risk.risk_index(lam, S1, S2s, mode))


def _dead_peer_worker(rank, world, port, outq):
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OPENBLAS_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        os._exit(0)                                     # leaves between steps, never joins the merge
    try:
        shard.merge_severity(np.zeros(16, np.uint8))
        outq.put("merged")
    except Exception as e:                              # the collective ends with an error, not a hang
        outq.put("error " + type(e).__name__)
    outq.close()
    outq.join_thread()
    os._exit(0)


def test_a_rank_that_leaves_ends_the_merge_with_an_error():
    """Failure detection of the sharded form on the host: when a rank exits before the
    severity merge, the surviving rank's collective fails within the process-group
    timeout instead of waiting forever."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dead_peer_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        msg = q.get(timeout=120)
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    assert msg.startswith("error"), msg
