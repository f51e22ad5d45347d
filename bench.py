#!/usr/bin/env python
"""Benchmark of the N-2 contingency screen (one JSON line on rank 0).

Workload (one step): the 118-bus synthetic study network (118 buses, 186
branches, 54 generators; seed 118 + rank), every unordered pair of its 240
outage elements (28,680 N-2 scenarios) at both load levels (70 % and 90 %) --
57,360 N-2 scenarios -- plus the 480 N-1 scenarios the Risk Index needs, and
the Risk Index of both levels.  Every scenario runs islanding, the
interior-point AC-OPF (FP64) and the small-signal eigen screen on the GPU.  The
headline is the mixed form (FP32 eigen screen, FP64 re-run in the guard band);
the FP64 form is measured on the same workload next to it.

value  = N-2 scenarios per second over all ranks, inputs resident in HBM,
         per-step time from CUDA events on the launching stream, L2 flushed
         (a 512 MB write) between steps outside the timed events.
e2e    = the same metric through the host-buffer C ABI (cs_submit_contingencies
         / cs_poll / cs_risk_index), host<->device copies inside the timing.
Multi-GPU (torchrun): each rank screens its own network replica (weak scaling,
no data-path collective); rank 0 prints the max-over-ranks time.

--impl reference times the CPU oracle (plain FP64, all host cores) on a bounded
sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "N-2 scenarios/s on 1 GB300 (mixed vs FP64 form, same accuracy); p50/p99 latency"
UNIT = "scenarios/s"
WORKLOAD = ("118-bus synthetic study network (118 buses, 186 branches, 54 generators), all 28,680 "
            "N-2 pairs of 240 elements x 2 load levels (70 %, 90 %) = 57,360 N-2 scenarios + 480 N-1, "
            "FP64 form, Risk Index of both levels")


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def _oracle_sample(net, n, seed):
    import numpy as np
    from paper_2512_08465_gb300 import synth
    rng = np.random.Generator(np.random.PCG64(seed))
    E = net.n_elem
    ii, jj = synth.all_pairs(E)
    ks = rng.choice(ii.size, size=n, replace=False)
    return [(int(q % 2), int(ii[k]), int(jj[k])) for q, k in enumerate(ks)]


def cpu_baseline(net, n=256, seed=1234, keep=False):
    """The oracle as it stands on a bounded sample of the workload, all host cores.
    keep: also return the oracle's records of that sample and of the N-1 branch set at
    the 70 % level (evaluated after the timing), for the per-output error table."""
    from oracle import pipeline
    cores = os.cpu_count() or 1
    sample = _oracle_sample(net, n, seed)
    t0 = time.perf_counter()
    recs = pipeline.evaluate_many(net, sample, cores)
    dt = time.perf_counter() - t0
    out = {"value": n / dt, "unit": UNIT, "cores": cores, "per_core": n / dt / cores, "kind": "oracle",
           "sample": f"{n} N-2 scenarios drawn uniformly (seed {seed}) from the 57,360 of the workload, "
                     f"half per load level; {dt:.1f} s wall on {cores} processes"}
    if not keep:
        return out
    n1 = [(0, e, -1) for e in range(net.n_branch)]
    return out, {"pairs": (sample, recs), "n1": (n1, pipeline.evaluate_many(net, n1, cores))}


# relative errors are taken against max(|reference|, floor), the floor being the absolute
# tolerance of the quantity (an angle or a real part near zero has no relative error)
REL_FLOOR = {"Vm": 1e-8, "Va": 1e-8, "cost": 1.0, "max_re": 1e-6, "min_zeta": 1e-6}


def _error_table(refs, got, nb):
    """Error of GPU records against the oracle's records of the same scenarios, per output:
    max and 99th percentile of the absolute and of the relative error of Vm and Va (every
    bus of every scenario whose OPF converged), OPF cost, max Re and min damping ratio
    (scenarios whose eigen screen ran), and the count of differing classes."""
    import numpy as np
    cols = {k: [] for k in ("Vm", "Va", "cost", "max_re", "min_zeta")}
    refv = {k: [] for k in cols}
    mism = 0
    for q, r in enumerate(refs):
        if int(got["klass"][q]) != int(r["klass"]):
            mism += 1
            continue
        if r.get("converged") and r.get("Vm") is not None:
            for k in ("Vm", "Va"):
                ref = np.asarray(r[k], dtype=np.float64)
                cols[k].append(got[k][q * nb:(q + 1) * nb] - ref)
                refv[k].append(ref)
            cols["cost"].append(np.array([got["cost"][q] - r["cost"]]))
            refv["cost"].append(np.array([r["cost"]]))
        if r["klass"] in (0, 4, 5):
            for k in ("max_re", "min_zeta"):
                cols[k].append(np.array([got[k][q] - r[k]]))
                refv[k].append(np.array([r[k]]))
    table = {"class_mismatches": mism, "scenarios": len(refs),
             "relative_error_floor": dict(REL_FLOOR)}
    for k in cols:
        if not cols[k]:
            table[k] = None
            continue
        d = np.abs(np.concatenate(cols[k]))
        ref = np.abs(np.concatenate(refv[k]))
        rel = d / np.maximum(ref, REL_FLOOR[k])
        table[k] = {"n": int(d.size), "max_abs": float(d.max()), "p99_abs": float(np.percentile(d, 99)),
                    "max_rel": float(rel.max()) if rel.size else None,
                    "p99_rel": float(np.percentile(rel, 99)) if rel.size else None}
    return table


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    from paper_2512_08465_gb300 import synth
    net = synth.case118()
    per_step = max(16, int(args.ref_sample))
    for w in range(args.warmup):
        cpu_baseline(net, n=min(per_step, 32), seed=100 + w)
    times = []
    last = None
    for k in range(args.steps):
        t0 = time.perf_counter()
        last = cpu_baseline(net, n=per_step, seed=1000 + k)
        times.append(time.perf_counter() - t0)
    mean = sum(times) / len(times)
    v = per_step / mean
    cores = os.cpu_count() or 1
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * mean,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + f"; reference arm: each step a bounded sample of {per_step} "
                                              f"N-2 scenarios of it on the host cores"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "per_core": v / cores, "kind": "oracle",
                             "sample": last["sample"] if last else ""},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, val in zip(names, r[5:9]):
                    if val.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _algorithmic_flops(net, res_lv, E, mixed_reruns=0):
    """Algorithmic FP64/FP32 work of the small-signal kernel for one step:
    10 n^3 flops per converged scenario (Golub & Van Loan's count for
    Hessenberg + Francis QR, eigenvalues only), n = 5 in-service generators - 1."""
    import numpy as np
    from paper_2512_08465_gb300 import synth
    ii, jj = synth.all_pairs(E)
    gout = (ii >= net.n_branch).astype(np.int64) + (jj >= net.n_branch).astype(np.int64)
    tot = 0.0
    for k in res_lv:
        ok = (k == 0) | (k == 4) | (k == 5) | (k == 6)
        nst = 5.0 * (net.n_gen - gout[ok]) - 1.0
        tot += float(np.sum(10.0 * nst ** 3))
    return tot


def _opf_flops_per_iter(st):
    """Algorithmic FP64 flops of one interior-point iteration, from the sizes of
    the network's symbolic analysis (cs_network_stats): block factorisation
    (each 4x4 block update and each L = U D^-1 block is 64 FMA, each pivot
    inverse ~200 flops), one block solve (two 4x4 mat-vecs per L block, one per
    pivot), one residual with its backward error (one 4x4 mat-vec per stored
    block, both triangles), and the branch flows with their first and second
    derivatives (~1,200 flops per branch)."""
    nb, nl, nu, nbr = st["n_bus"], st["l_blocks"], st["block_updates"], st["n_branch"]
    factor = nu * 128 + nl * 128 + nb * 200
    solve = 2 * nl * 32 + nb * 32
    residual = (2 * nl + nb) * 32
    return factor + solve + residual + nbr * 1200


# DRAM traffic of a kernel group per processed unit, from the committed ncu summary of
# its dominant kernel: a line "traffic: <group> <sha16 of the kernel source> <bytes per
# unit>" in profiles/.  Reported only while the kernel source still has that hash (a
# capture of an older kernel is not the traffic of this build).
_TRAFFIC_SRC = {"opf": "paper_2512_08465_gb300/csrc/k_opf.cu", "dyn": "paper_2512_08465_gb300/csrc/k_dyn.cu"}


def _captured_traffic(group, units_per_launch):
    import glob
    import hashlib
    import re
    src = os.path.join(ROOT, _TRAFFIC_SRC[group])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    found = None
    for fn in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for m in re.finditer(r"^traffic: (\w+) ([0-9a-f]{16}) ([0-9.eE+]+)\s*$", open(fn).read(), re.M):
            if m.group(1) == group:
                found = (m.group(2), float(m.group(3)), os.path.basename(fn))
    if found is None:
        return {"traffic": None, "traffic_source": "no ncu capture of this kernel group in profiles/"}
    if found[0] != sha:
        return {"traffic": None, "traffic_source": f"profiles/{found[2]}: captured on an earlier version of "
                                                   f"{_TRAFFIC_SRC[group]} (source hash {found[0]}, now {sha})"}
    return {"traffic": found[1] * units_per_launch,
            "traffic_source": f"profiles/{found[2]}: ncu dram__bytes_read.sum + dram__bytes_write.sum per "
                              f"unit ({found[1]:.4g} B) x the units of an average launch of this step"}


def run_ours(args):
    import numpy as np
    rank, world, local = _env_rank()
    cpu = recs = None
    if rank == 0 and not args.no_cpu_baseline:
        from paper_2512_08465_gb300 import synth as _s
        cpu, recs = cpu_baseline(_s.case118(), n=args.cpu_sample, keep=True)   # spawned workers, before any GPU call
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2512_08465_gb300 import cs, shard, synth
    net = synth.case118()                                 # one network, its scenarios sharded over the ranks
    E = net.n_elem
    npair = E * (E - 1) // 2
    lam = synth.failure_rates(E, 2512)
    lam_d = torch.as_tensor(lam, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # this rank's contiguous block of the pairs and of the single outages of each level
    p0, pc = shard.pair_block(rank, world, npair)
    s0, sc_ = shard.pair_block(rank, world, E)

    def make(prec, **opt):
        ctx = cs.Context(device=local, precision=prec, **opt)
        nid = ctx.load_network(net)
        return ctx, nid

    ei_all = torch.empty(npair, dtype=torch.int32, device=dev)
    ej_all = torch.empty(npair, dtype=torch.int32, device=dev)
    cs.enumerate_pairs_device(E, 0, npair, ei_all, ej_all)
    ei, ej = ei_all[p0:p0 + pc], ej_all[p0:p0 + pc]
    n1i = torch.arange(s0, s0 + sc_, dtype=torch.int32, device=dev)
    n1j = torch.full((sc_,), -1, dtype=torch.int32, device=dev)
    # severity tables of both levels in one buffer: [S1 (E) | S2 (npair)] per level; after
    # each rank fills its block, one element-wise MIN over the ranks merges them (255 = not
    # evaluated), and the exact Risk Index of the merged tables is the single-rank one
    flat = torch.empty(2 * (E + npair), dtype=torch.uint8, device=dev)
    tabs = {lv: (flat[lv * (E + npair):lv * (E + npair) + E], flat[lv * (E + npair) + E:(lv + 1) * (E + npair)])
            for lv in (0, 1)}
    R = {lv: torch.empty(E, dtype=torch.float64, device=dev) for lv in (0, 1)}

    def measure(ctx, nid, warmup, steps, clocks=False, main=False):
        outs = {lv: (ctx.alloc_results(pc, dev, main_island=main), ctx.alloc_results(sc_, dev, main_island=main))
                for lv in (0, 1)}
        launches = [0]

        def step():
            for lv in (0, 1):
                ctx.evaluate_device(nid, lv, ei, ej, outs[lv][0], stream)
                launches[0] += ctx.last_launch_count()
                ctx.evaluate_device(nid, lv, n1i, n1j, outs[lv][1], stream)
                launches[0] += ctx.last_launch_count()
            flat.fill_(shard.MISSING)
            for lv in (0, 1):
                tabs[lv][1][p0:p0 + pc].copy_(outs[lv][0]["severe"])
                tabs[lv][0][s0:s0 + sc_].copy_(outs[lv][1]["severe"])
            shard.merge_severity_device(flat)
            for lv in (0, 1):
                cs.risk_reduce_device(E, tabs[lv][0], tabs[lv][1], lam_d, R[lv], cs.RISK_ORDERED, stream)
                launches[0] += 1

        for _ in range(warmup):
            step()
        ctx.sync(stream)
        torch.cuda.synchronize()
        launches[0] = 0
        ctx.set_timing(True)
        sampler = ClockSampler(local) if clocks else None
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        wall0 = time.perf_counter()
        step_ms = []
        for _ in range(steps):
            flush.zero_()                                   # L2 flush, outside the timed events
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        clk = sampler.stop() if sampler else None
        ctx.sync(stream)
        kms, kcnt = ctx.kernel_times()
        ctx.set_timing(False)
        ms = sum(step_ms) / len(step_ms)
        ms_max = shard.max_over_ranks(ms, device=dev)            # the slowest rank sets the step
        if world > 1:
            torch.distributed.barrier()
        klass = [outs[lv][0]["klass"].cpu().numpy() for lv in (0, 1)]
        stats = {f: [outs[lv][0][f].cpu().numpy() for lv in (0, 1)] for f in ("max_re", "min_zeta")}
        iters = sum(int(outs[lv][q]["opf_iters"].to(torch.int64).sum().item()) for lv in (0, 1) for q in (0, 1))
        mk = [outs[lv][0]["main_klass"].cpu().numpy() for lv in (0, 1)] if main else None
        shed = [outs[lv][0]["shed_mw"].cpu().numpy() for lv in (0, 1)] if main else None
        # the merged tables' Risk Index against the context's own (one rank: the same tables)
        r_same = None
        if world == 1:
            r_same = all(np.array_equal(R[lv].cpu().numpy(), ctx.risk_index(nid, lv, lam, cs.RISK_ORDERED)[0])
                         for lv in (0, 1))
        rsha = __import__("hashlib").sha256(b"".join(R[lv].cpu().numpy().tobytes() for lv in (0, 1))).hexdigest()[:16]
        return dict(ms=ms_max, wall=wall, kms=kms, kcnt=kcnt, clocks=clk, launches=launches[0],
                    klass=klass, iters=iters, stats=stats, main_klass=mk, shed=shed, r_same=r_same, r_sha=rsha)

    def accuracy(ctx, nid):
        """Error table of this form against the oracle's records (rank 0, after the timing)."""
        out = {}
        for name, (sc, refs) in recs.items():
            by_lv = {}
            for q, (lv, i, j) in enumerate(sc):
                by_lv.setdefault(lv, []).append(q)
            got = {}
            for lv, qs in by_lv.items():
                ti = torch.as_tensor(np.array([sc[q][1] for q in qs], np.int32), device=dev)
                tj = torch.as_tensor(np.array([sc[q][2] for q in qs], np.int32), device=dev)
                o = ctx.alloc_results(len(qs), dev, net.n_bus)
                ctx.evaluate_device(nid, lv, ti, tj, o, stream)
                ctx.sync(stream)
                g = {k: v.cpu().numpy() for k, v in o.items()}
                for k, v in g.items():
                    got.setdefault(k, np.zeros(len(sc) * (net.n_bus if k in ("Vm", "Va") else 1), v.dtype))
                    for m, q in enumerate(qs):
                        if k in ("Vm", "Va"):
                            got[k][q * net.n_bus:(q + 1) * net.n_bus] = v[m * net.n_bus:(m + 1) * net.n_bus]
                        else:
                            got[k][q] = v[m]
            out[name] = _error_table(refs, got, net.n_bus)
        return out

    ctx_m, nid_m = make(cs.PREC_MIXED)
    mixed = measure(ctx_m, nid_m, args.warmup, args.steps, clocks=True)
    reruns_m = ctx_m.eigen_reruns()
    # Monte-Carlo Risk Index (uncertain failure rates): 10,000 seeded rate vectors against the
    # level-0 tables of this step, exact per sample; outside the timed step
    gen = torch.Generator(device=dev).manual_seed(2512)
    lam_mc = 0.01 + 0.99 * torch.rand((10000, E), dtype=torch.float64, device=dev, generator=gen)
    r_mc = torch.empty_like(lam_mc)
    ctx_m.risk_index_batch(nid_m, 0, lam_mc, r_mc, cs.RISK_ORDERED, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx_m.risk_index_batch(nid_m, 0, lam_mc, r_mc, cs.RISK_ORDERED, stream)
    e1.record(stream)
    e1.synchronize()
    ctx_m.sync(stream)
    mc_ms = e0.elapsed_time(e1)
    mc = {"samples": int(lam_mc.shape[0]), "elements": E, "ms": mc_ms,
          "samples_per_s": lam_mc.shape[0] / (mc_ms / 1e3),
          "R_p50_p95_of_max_element": [float(x) for x in torch.quantile(r_mc.max(dim=1).values,
                                                                          torch.tensor([0.5, 0.95], device=dev,
                                                                                       dtype=torch.float64)).cpu()]}
    del lam_mc, r_mc
    ctx_d, nid_d = make(cs.PREC_FP64)
    fp64 = measure(ctx_d, nid_d, 1, args.steps)
    same = all(np.array_equal(a, b) for a, b in zip(mixed["klass"], fp64["klass"]))
    # largest deviation of the mixed form's eigen statistics from the FP64 form's (FP32 screen
    # refined in FP64 outside the guard band; scenarios re-run in FP64 agree to rounding)
    mdev = {}
    for f in ("max_re", "min_zeta"):
        d = [np.abs(a - b)[np.isfinite(a) & np.isfinite(b)] for a, b in zip(mixed["stats"][f], fp64["stats"][f])]
        mdev[f] = float(max((x.max() if x.size else 0.0) for x in d))
    acc = None
    if rank == 0 and recs is not None:
        acc = {"mixed": accuracy(ctx_m, nid_m), "fp64": accuracy(ctx_d, nid_d),
               "sets": {"n1": f"the {net.n_branch} branch N-1 scenarios at the 70 % level",
                        "pairs": f"the {args.cpu_sample} sampled N-2 scenarios of the CPU baseline"}}
    ctx_d.close()
    # main-island form: every islanded pair also gets its main island's OPF (classes unchanged)
    ctx_i, nid_i = make(cs.PREC_MIXED, main_island=1)
    isl = measure(ctx_i, nid_i, 1, min(2, args.steps), main=True)
    ctx_i.close()
    mk = np.concatenate(isl["main_klass"])
    shed = np.concatenate(isl["shed"])
    n_isl = int((mk != 255).sum())
    main_form = {"value": 2 * npair / (isl["ms"] / 1e3), "ms_per_step": isl["ms"], "steps": min(2, args.steps),
                 "kernel_ms_per_step": {k: v / min(2, args.steps) for k, v in isl["kms"].items()},
                 "classes_identical_to_mixed": bool(all(np.array_equal(a, b) for a, b in
                                                        zip(mixed["klass"], isl["klass"]))),
                 "main_island_opfs_per_step": n_isl,
                 "main_klass_counts": {name: int((mk == code).sum()) for code, name in
                                       ((0, "secure"), (2, "opf_nonconv"), (3, "limit"), (4, "ss_unstable"),
                                        (5, "ss_poorly_damped"), (6, "eig_fail"))},
                 "shed_mw_mean_over_islanded": float(shed[mk != 255].mean()) if n_isl else None}

    n2 = 2 * npair
    value = n2 / (mixed["ms"] / 1e3)
    kms, kcnt = mixed["kms"], mixed["kcnt"]
    share = {k: v / max(1e-9, sum(kms.values())) for k, v in kms.items()}
    # Roofline of both kernel groups; the one with more device time per step is the
    # "roofline" entry.  Chunks on two streams overlap, so each launch's duration
    # includes time shared with the other group's kernels.
    peak64, peak32 = cs.alu_peak(local)
    fl = _opf_flops_per_iter(ctx_m.network_stats(nid_m))
    roofs = {
        "opf": {"kernel": "opf_kernel (interior-point OPF: branch derivatives, block LDL^T, refined solves)",
                "bound": "alu", "unit": "TFLOP/s", "peak": peak64,
                "peak_source": "measured in this run: FP64 FMA-chain probe (cs_alu_peak), all SMs",
                "work": "per interior-point iteration: block factorisation + one block solve + one residual "
                        "+ branch derivatives, counted from the symbolic analysis (cs_network_stats), times the "
                        "iterations each scenario took",
                "achieved": mixed["iters"] * fl / (kms["opf"] / args.steps / 1e3) / 1e12,
                "iterations_per_step": mixed["iters"], "flops_per_iteration": fl},
        "dyn": {"kernel": "small-signal kernels (model + balancing; cluster Hessenberg; shared-memory Francis QR; "
                          "FP64 refinement; FP64 re-run)", "bound": "alu", "unit": "TFLOP/s", "peak": peak32,
                "peak_source": "measured in this run: FP32 FMA-chain probe (cs_alu_peak), all SMs",
                "work": "10 n^3 flops per converged scenario, n = 5 x in-service generators - 1",
                "achieved": _algorithmic_flops(net, mixed["klass"], E) / (kms["dyn"] / args.steps / 1e3) / 1e12},
    }
    n_opf = sum(int(np.sum(k != 1)) for k in mixed["klass"])
    n_conv = sum(int(np.sum((k == 0) | (k == 4) | (k == 5) | (k == 6))) for k in mixed["klass"])
    units = {"opf": n_opf, "dyn": n_conv}
    for k, r in roofs.items():
        launches = max(1.0, kcnt[k] / args.steps)
        r.update({"launches_per_step": kcnt[k] / args.steps, "avg_launch_ms": kms[k] / max(1, kcnt[k])})
        r.update(_captured_traffic(k, units[k] / launches))
    # opf_kernel is the dominant single kernel of the step (about half of the serialised
    # launch list; profiles/launch_list_118bus_n2_step.md); the small-signal group's five
    # kernels are reported beside it
    roof = roofs["opf"]
    roof_other = roofs["dyn"]

    # ---- end to end through the host-buffer ABI (mixed form), this rank's block ----
    ei_h = ei.cpu().numpy()
    ej_h = ej.cpu().numpy()
    n1i_h = n1i.cpu().numpy()
    n1j_h = n1j.cpu().numpy()
    chunk = args.request
    lat = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pend = []
    for lv in (0, 1):
        for c0 in range(0, pc, chunk):
            rid = ctx_m.submit(nid_m, lv, ei_h[c0:c0 + chunk], ej_h[c0:c0 + chunk])
            pend.append((rid, time.perf_counter()))
        pend.append((ctx_m.submit(nid_m, lv, n1i_h, n1j_h), time.perf_counter()))
    for rid, ts in pend:
        ctx_m.poll(rid, 600_000_000)
        lat.append(1e3 * (time.perf_counter() - ts))
    for lv in (0, 1):
        ctx_m.risk_index(nid_m, lv, lam, cs.RISK_ORDERED)
    e2e_step = shard.max_over_ranks(1e3 * (time.perf_counter() - t0), device=dev)
    h2d = 2 * (2 * pc + 2 * sc_) * 4 + 2 * E * 8
    d2h = 2 * (pc + sc_) * (1 + 1 + 1 + 2 + 2 + 8 * 6) + 2 * E * 8   # every per-scenario record field + R
    lat.sort()
    ctx_m.close()
    # ---- serving phase: Poisson arrivals over two resident networks, both forms ----
    serving = None
    if rank == 0 and not args.no_serve:
        serving = {name: serve_phase(prec, args.serve_requests, args.serve_burst, args.serve_seed)
                   for name, prec in (("mixed", cs.PREC_MIXED), ("fp64", cs.PREC_FP64))}

    if rank == 0:
        for r in (roof, roof_other):
            r["frac"] = r["achieved"] / r["peak"] if r.get("achieved") is not None else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mixed["ms"], "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("FP64 form", "mixed form (FP64 OPF; FP32 eigen screen with "
                                                               "FP64 refinement of the decisive eigenvalues and "
                                                               "FP64 re-run in the guard band)"),
                       "form": "mixed", "network_seed": 118, "n2_scenarios_per_step": n2,
                       "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"pair range sharded over {world} rank(s), severity tables merged by one "
                                      f"element-wise MIN all-reduce" if world > 1 else "one GPU",
                       "wall_s_timed_region": mixed["wall"], "eigen_fp64_reruns_per_step":
                           (reruns_m / (args.warmup + args.steps)) if args.warmup + args.steps else None},
            "fp64_form": {"value": n2 / (fp64["ms"] / 1e3), "ms_per_step": fp64["ms"],
                          "kernel_ms_per_step": {k: v / args.steps for k, v in fp64["kms"].items()},
                          "classes_identical_to_mixed": bool(same),
                          "mixed_max_abs_dev": mdev},
            "risk_index": {"merged_tables_equal_context_tables": mixed["r_same"], "sha16": mixed["r_sha"],
                           "sha16_fp64_form": fp64["r_sha"]},
            "accuracy_vs_oracle": acc,
            "main_island_form": main_form,
            "roofline": roof,
            "roofline_other": roof_other,
            "risk_index_monte_carlo": mc,
            "kernel_ms_per_step": {k: v / args.steps for k, v in kms.items()},
            "kernel_share": share,
            "e2e": {"value": n2 / (e2e_step / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_step,
                    "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                                   "request_scenarios": chunk, "requests": len(lat),
                                   "note": "requests submitted together; the serving entry has Poisson arrivals"}},
            "serving": serving,
            "gpu_launches": mixed["launches"],
            "clocks": mixed["clocks"],
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_profile(args):
    """Small fixed case for profiler captures (kernels as in the benchmark)."""
    import torch
    from paper_2512_08465_gb300 import cs, synth
    dev = torch.device("cuda", 0)
    net = synth.case118()
    ctx = cs.Context(precision=cs.PREC_FP64 if args.fp64 else cs.PREC_MIXED)
    nid = ctx.load_network(net)
    E = net.n_elem
    n = min(args.profile, E * (E - 1) // 2)
    ei = torch.empty(n, dtype=torch.int32, device=dev)
    ej = torch.empty(n, dtype=torch.int32, device=dev)
    cs.enumerate_pairs_device(E, 0, n, ei, ej)
    out = ctx.alloc_results(n, dev)
    for rep in range(2):
        if rep == 1:
            ctx.set_timing(True)
        ctx.evaluate_device(nid, 0, ei, ej, out)
        ctx.sync()
    kms, kcnt = ctx.kernel_times()
    k = out["klass"].cpu().numpy()
    print(json.dumps({"profile_pairs": n, "kernel_ms": kms, "launches": kcnt,
                      "classes": {int(c): int((k == c).sum()) for c in set(k.tolist())}}))
    ctx.close()


def serve_phase(prec, n_requests, n_burst, seed):
    """Serving form: Poisson arrivals of requests over several resident networks
    (the 118-bus study network, both levels, and a 300-bus network of the same
    construction), each request a log-uniform number in [16, 4096] of random
    branch pairs of a uniformly drawn network and level.  The saturation
    throughput is measured first with a burst of requests submitted at once;
    then, for offered loads of 0.25, 0.5 and 0.9 of it, requests arrive at
    exponential intervals and each one's latency (submit to completed poll,
    host clock) is recorded.  Host-buffer ABI, precision form `prec`."""
    import math
    import numpy as np
    import torch  # noqa: F401  (CUDA context in this process before the library's threads)
    from paper_2512_08465_gb300 import cs, synth
    specs = [("118-bus", synth.case118()), ("300-bus", synth.case_scaled(300, seed=300, vband=(0.85, 1.15)))]
    ctx = cs.Context(precision=prec)
    t0 = time.perf_counter()
    ids = [ctx.load_network(net) for _, net in specs]
    load_s = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    pairs = [synth.all_pairs(net.n_branch) for _, net in specs]

    def draw():
        k = int(rng.integers(len(specs)))
        lv = int(rng.integers(len(specs[k][1].levels)))
        m = int(round(math.exp(rng.uniform(math.log(16), math.log(4096)))))
        ii, jj = pairs[k]
        sel = rng.choice(ii.size, m, replace=False)
        return k, lv, ii[sel], jj[sel]

    def run(reqs, arrivals):
        """Submit reqs at the given offsets (s) and poll; latency per request."""
        pend, lat, done_sc = {}, [], 0
        q, t_start = 0, time.perf_counter()
        while q < len(reqs) or pend:
            now = time.perf_counter() - t_start
            while q < len(reqs) and arrivals[q] <= now:
                k, lv, ei, ej = reqs[q]
                pend[ctx.submit(ids[k], lv, ei, ej)] = (time.perf_counter(), ei.size)
                q += 1
            for rid in list(pend):
                if ctx.poll(rid, 0) is not None:
                    ts, m = pend.pop(rid)
                    lat.append(time.perf_counter() - ts)
                    done_sc += m
            time.sleep(0.0002)
        return lat, done_sc, time.perf_counter() - t_start

    # warm-up, then saturation: every request of a burst submitted at once
    run([draw() for _ in range(4)], [0.0] * 4)
    burst = [draw() for _ in range(n_burst)]
    _, sc, wall = run(burst, [0.0] * len(burst))
    sat = sc / wall
    mean_size = float(np.mean([r[2].size for r in burst]))
    out = {"form": "mixed" if prec == cs.PREC_MIXED else "fp64",
           "networks": [{"name": n, "n_bus": net.n_bus, "n_branch": net.n_branch, "n_gen": net.n_gen,
                         "levels": len(net.levels), "state_order": 5 * net.n_gen - 1} for n, net in specs],
           "load_networks_s": load_s, "request_sizes": "log-uniform integers in [16, 4096], random branch pairs",
           "saturation": {"requests": len(burst), "scenarios": sc, "wall_s": wall, "scenarios_per_s": sat},
           "rates": []}
    for frac in (0.25, 0.5, 0.9):
        reqs = [draw() for _ in range(n_requests)]
        rate = frac * sat / mean_size                       # requests per second
        arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
        lat, sc, wall = run(reqs, arrivals)
        lat_ms = np.sort(np.array(lat)) * 1e3
        out["rates"].append({"offered_fraction": frac, "offered_requests_per_s": rate,
                             "requests": len(reqs), "scenarios": sc, "wall_s": wall,
                             "achieved_scenarios_per_s": sc / wall,
                             "latency_ms": {"p50": float(np.percentile(lat_ms, 50)),
                                            "p99": float(np.percentile(lat_ms, 99)),
                                            "max": float(lat_ms[-1])}})
    out["serving_stats"] = ctx.serving_stats()
    ctx.close()
    return out


def run_hessenberg(args):
    """--hessenberg N: the blocked Hessenberg reduction of the eigen screen of large networks
    (cs_hessenberg_tc: panels on the SIMT pipes, trailing updates on the tensor cores) on a
    batch of seeded N x N FP32 matrices (N = 2,499 is the state order of a 2000-bus network
    with 500 generators): time per matrix (CUDA events, inputs resident, after a warm-up),
    the reduction's algorithmic rate (10/3 N^3 flops per matrix) and the share of that work
    in the tensor-core products (the trailing updates: 2 N^3 / 3 of the right update plus
    4 N^3 / 3 of the left one, before the TF32 x 3 split)."""
    import torch
    from paper_2512_08465_gb300 import cs
    n, b = args.hessenberg, args.hessenberg_batch
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(2499)
    A0 = torch.randn(b, n, n, device=dev, generator=g)
    ctx = cs.Context()
    A = A0.clone()
    ctx.hessenberg_tc(A)                                   # warm-up (workspace, kernels)
    ctx.sync()
    times = []
    for _ in range(args.steps):
        A.copy_(A0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.hessenberg_tc(A)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ctx.sync()
    ms = sum(times) / len(times)
    flops = 10.0 / 3.0 * n ** 3 * b
    below = torch.tril(A, diagonal=-2).abs().max().item()
    fro = (torch.linalg.matrix_norm(A.double()) / torch.linalg.matrix_norm(A0.double())).max().item()
    print(json.dumps({"mode": "hessenberg", "n": n, "batch": b, "steps": args.steps, "ms_per_batch": ms,
                      "ms_per_matrix": ms / b, "algorithmic_tflops": flops / (ms / 1e3) / 1e12,
                      "tensor_core_share_of_flops": (2.0 / 3.0 + 4.0 / 3.0) / (10.0 / 3.0),
                      "max_below_subdiagonal": below, "frobenius_ratio_max": fro}))
    ctx.close()


def run_scale(args):
    """--scale K: the 2000-bus configuration on a seeded sample of K random N-2 branch pairs
    (network: 2,000 buses, 3,000 branches, 500 generators, state order 2,499; 0.85-1.15 p.u.
    voltage band as for the 300-bus network; interior-point cap 150 iterations, as its base-case
    OPF needs 70).  Mixed form (tensor-core Hessenberg reduction,
    FP32 QR, FP64 re-run in the guard band) and, on the first K/2 pairs, the FP64 form:
    scenarios/s, per-kernel-group device time, class mix, and the mixed form's deviation from
    the FP64 form on the common pairs.  Inputs resident; CUDA events on the launching stream."""
    import numpy as np
    import torch
    from paper_2512_08465_gb300 import cs, synth
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    net = synth.case_scaled(2000, seed=2000, vband=(0.85, 1.15))
    net.opf_max_it = 150                      # this network's cap (cs_network_desc.opf_max_it)
    ii, jj = synth.all_pairs(net.n_branch)
    rng = np.random.default_rng(200000)
    sel = np.sort(rng.choice(ii.size, args.scale, replace=False))
    ei = torch.as_tensor(ii[sel].astype(np.int32), device=dev)
    ej = torch.as_tensor(jj[sel].astype(np.int32), device=dev)
    out = {"mode": "scale", "network": {"n_bus": net.n_bus, "n_branch": net.n_branch, "n_gen": net.n_gen,
                                        "state_order": 5 * net.n_gen - 1},
           "pairs": int(args.scale), "pair_draw": "seeded uniform sample of the 4,498,500 branch pairs"}
    res = {}
    for name, prec, m in (("mixed", cs.PREC_MIXED, args.scale), ("fp64", cs.PREC_FP64, max(1, args.scale // 2))):
        ctx = cs.Context(precision=prec)
        tl = time.perf_counter()
        nid = ctx.load_network(net)
        load_s = time.perf_counter() - tl
        o = ctx.alloc_results(m, dev)
        ctx.set_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.evaluate_device(nid, 0, ei[:m], ej[:m], o)
        e1.record()
        e1.synchronize()
        ctx.sync()
        ms = e0.elapsed_time(e1)
        kms, _ = ctx.kernel_times()
        k = o["klass"].cpu().numpy()
        res[name] = {k2: v.cpu().numpy() for k2, v in o.items()}
        out[name] = {"scenarios": m, "ms": ms, "scenarios_per_s": m / (ms / 1e3), "load_network_s": load_s,
                     "kernel_ms": kms, "classes": {cs.CLASSES[c]: int((k == c).sum()) for c in range(7)},
                     "eigen_fp64_reruns": ctx.eigen_reruns()}
        ctx.close()
    m = out["fp64"]["scenarios"]
    a, b = res["fp64"], res["mixed"]
    ok = np.isfinite(a["max_re"][:m]) & np.isfinite(b["max_re"][:m])
    out["mixed_vs_fp64"] = {"classes_identical": bool(np.array_equal(a["klass"][:m], b["klass"][:m])),
                            "max_abs_dev_max_re": float(np.abs(a["max_re"][:m] - b["max_re"][:m])[ok].max())
                            if ok.any() else None,
                            "max_abs_dev_min_zeta": float(np.abs(a["min_zeta"][:m] - b["min_zeta"][:m])[ok].max())
                            if ok.any() else None}
    out["wall_s"] = time.perf_counter() - t0
    print(json.dumps(out))


def run_serve(args):
    """--serve: the serving phase alone, both forms, with the larger request counts."""
    from paper_2512_08465_gb300 import cs
    out = {"mode": "serve", "metric": "N-2 scenarios/s and request latency under Poisson load",
           "unit": "scenarios/s",
           "forms": [serve_phase(p, args.serve_requests, args.serve_burst, args.serve_seed)
                     for p in (cs.PREC_MIXED, cs.PREC_FP64)]}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--ref-sample", type=int, default=96)
    ap.add_argument("--cpu-sample", type=int, default=256)
    ap.add_argument("--request", type=int, default=4096, help="scenarios per request in the e2e leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64", action="store_true", help="--profile: run the FP64 form instead of the mixed one")
    ap.add_argument("--serve", action="store_true",
                    help="serving form: Poisson request arrivals over several networks, p50/p99 latency")
    ap.add_argument("--serve-requests", type=int, default=24, help="serving phase: requests per offered load")
    ap.add_argument("--serve-burst", type=int, default=16, help="serving phase: requests of the saturation burst")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving phase of the default run")
    ap.add_argument("--serve-seed", type=int, default=2024)
    ap.add_argument("--profile", type=int, default=0, metavar="N",
                    help="profiling case for ncu: N pairs of the 70 %% level, one warm-up and one launch set, "
                         "no baseline, no e2e, prints per-kernel times")
    ap.add_argument("--hessenberg", type=int, default=0, metavar="N",
                    help="time the tensor-core blocked Hessenberg reduction on N x N matrices")
    ap.add_argument("--hessenberg-batch", type=int, default=8)
    ap.add_argument("--scale", type=int, default=0, metavar="K",
                    help="2000-bus configuration on K seeded random branch pairs (mixed and FP64 forms)")
    args = ap.parse_args()
    if args.scale:
        run_scale(args)
        return
    if args.hessenberg:
        run_hessenberg(args)
        return
    if args.profile:
        run_profile(args)
        return
    if args.serve:
        run_serve(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
