#!/usr/bin/env python3
"""Queue throughput benchmark (one JSON line on stdout).

Workload (one step): the pairwise 50/50 interleaved schedule at its largest
size, 2^20 threads x 100 operations, capacity 2^20 uint64 slots, seed 0: op i
of thread t is an enqueue of token (t << 32) | (seq + 1) or a dequeue, as the
seeded bit schedule says.  One step resets and runs every queue kind (G-LFQ,
G-WFQ, G-WFQ-YMC) once; the metric is successful (enqueue + dequeue)
operations per second over the step (Section V-A throughput metric).

Also reported:
  roofline     the dominant run kernel's algorithmic L2 atomics per second
               against the same-box measured warp-coalesced 64-bit CAS rate
  e2e          the same metric through the public batch API with host buffers
               (pinned host -> device copy of the items, enqueue batch,
               dequeue batch, device -> host copy of the results)
  cpu_baseline the oracle's mutex-guarded std::deque on the host cores
  sweep        kernel-only Mops/s per queue for 2^10 .. 2^20 threads
  phases       enqueue-only then dequeue-only phases (min(2^20, T x ops) items)

--impl reference times the oracle's mutex deque (the CPU reference arm).
Multi-GPU: independent replicas, one per rank, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queue Mops/s (enq+deq) vs threads; % of measured L2-atomic peak; serving p99"
CAPACITY = 1 << 20
# DRAM bytes (read + write) per launch of each run kernel at the headline size, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum, one kernel, one launch; profiles/
# traffic_k_run_mixed_2p18.md).  G-WFQ: captured at the headline size itself (`bench.py
# --no-sweep --no-e2e --no-cpu --no-apps --no-batched --no-serving --kinds wfq --steps 1
# --warmup 1`; a one-pass metric set): 391.11 + 113.24 MB as ncu printed them.  G-WFQ-YMC: its
# 2^18-thread case (`... --threads 262144 --kinds ymc`), 240533760 + 156694272 bytes for 26.2 M
# operations (each ticket's cell touched once, so the bytes grow with the operations), scaled by
# the 4x operations of the headline launch.  G-LFQ's traffic is its workspace read once and does
# not grow with the operations; it has no headline-size capture.  Set an entry to None whenever
# that kernel changes.
E2E_THREADS = 1 << 17   # records of the e2e queues (threads of their batch kernels)
NCU_TRAFFIC = {"lfq": None, "wfq": 391110000 + 113240000, "ymc": 4 * (240533760 + 156694272)}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--threads", type=int, default=1 << 20)
    p.add_argument("--ops", type=int, default=100)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--kinds", default=None, help="comma list of queue kinds (default: all implemented)")
    p.add_argument("--no-sweep", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-threads", type=int, default=1 << 19,
                   help="logical threads in the CPU sample (2^19 x 100 ops: about 10 s on the 16 host cores)")
    p.add_argument("--no-apps", action="store_true", help="skip the application measurements (BFS, ray tracing)")
    p.add_argument("--no-batched", action="store_true", help="skip the batched / persistent / graph comparisons")
    p.add_argument("--no-serving", action="store_true", help="skip the BFS serving measurements")
    return p.parse_args()


ALL_KINDS = ["lfq", "wfq", "ymc"]


def workload_config(args, kinds, world):
    """The `config` object of both arms: the workload this line measures."""
    T, K = args.threads, args.ops
    return {"workload": "pairwise 50/50 interleaved by seed, %d threads x %d ops, capacity 2^20 uint64, queues %s"
                        % (T, K, "+".join(kinds)),
            "threads": T, "ops_per_thread": K, "capacity": CAPACITY, "ymc_pool_cells": int(1.25 * T * K) + (1 << 21),
            "block": 256, "seed": args.seed, "parallelism": "replicas" if world > 1 else "single",
            "l2": "flushed between timed steps (256 MiB write); queue state re-initialised inside each step"}


def replica_totals(total_ms, succ_ops, device=None):
    """Replicas (one independent queue set per rank, no data exchange): the job's
    time is the slowest rank's and its operations are the sum over ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), float(succ_ops)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([float(succ_ops)], dtype=torch.float64, device=device)
    dist.all_reduce(s)
    return float(t.item()), float(s.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", str(device_index)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self, window=None):
        """Median SM clock and throttle reasons of the samples taken inside
        `window` (host epoch seconds, start and end of the timed region)."""
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        import datetime
        rows = []
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        inside = [r for r in rows if window and window[0] <= r[0] <= window[1]]
        use = inside or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = {nm for r in use for nm, v in zip(names, r[3]) if v.lower().startswith("active")}
        sm = [r[1] for r in use]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(r[2] for r in use) if use else None,
                "samples": len(sm), "samples_in_timed_region": len(inside), "reasons": sorted(reasons)}


def cpu_baseline(T, K, seed, cpu_threads):
    import oracle
    Ts = min(T, cpu_threads)
    sched = __import__("synth").mixed_schedule_bits(seed, Ts, K)
    cores = os.cpu_count() or 1
    secs, c, nt = oracle.mutex_run(1, Ts, K, sched=sched, nthreads=cores)
    succ = int(c[0] + c[2])
    return {"value": succ / secs / 1e6, "unit": "Mops/s", "cores": nt, "kind": "oracle",
            "sample": "mutex-guarded std::deque, same 50/50 schedule, first %d of %d threads x %d ops "
                      "(%d ops, %.2f s)" % (Ts, T, K, Ts * K, secs)}


def bench_apps(gq, synth, kinds, dev, reps=3):
    """Applications on each queue kind, outside the headline step: level-synchronous
    BFS over two frontier queues (R-MAT scale 22 from vertex 0, 4096 x 4096 grid
    from its corner; ms and scanned edges per second) and tile-queue wavefront
    ray tracing (MRays/s = traced segments per second)."""
    import torch
    out = {}
    graphs = {"rmat22": synth.rmat_csr_fast(22, seed=0), "grid4096": synth.grid_csr(4096, 4096)}
    for gname, (off, adj) in graphs.items():
        n = len(off) - 1
        d_off = torch.from_numpy(off.view(np.int64)).to(dev)
        d_adj = torch.from_numpy(adj.view(np.int32)).to(dev)
        dist = torch.empty(n, dtype=torch.int32, device=dev)
        stats = torch.zeros(4, dtype=torch.int64, device=dev)
        levels_hint = 8192 if gname.startswith("grid") else 64
        for k in kinds:
            if k == "ymc":
                cap = 3 * n + 64 * (levels_hint + 1) + (1 << 16)
            else:
                cap = min(1 << max(12, (n - 1).bit_length()), 1 << 23)
            qa, qb = gq.Queue(k, cap, 4, 1 << 19), gq.Queue(k, cap, 4, 1 << 19)
            gq.gq_bfs(qa.handle, qb.handle, d_off, d_adj, 0, dist, stats)
            torch.cuda.synchronize()
            ms = []
            for _ in range(reps):
                qa.reset()
                qb.reset()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                gq.gq_bfs(qa.handle, qb.handle, d_off, d_adj, 0, dist, stats)
                e1.record()
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            st = stats.cpu().numpy()
            assert qa.sync_status() == 0 and qb.sync_status() == 0 and st[3] == 0
            t = float(np.median(ms))
            out["bfs_%s_%s" % (gname, k)] = {"ms": round(t, 3), "levels": int(st[0]), "reached": int(st[1]),
                                              "edges_scanned": int(st[2]),
                                              "gteps": round(float(st[2]) / (t * 1e-3) / 1e9, 3)}
            qa.close()
            qb.close()
    # wavefront ray tracing: 1920 x 1080, 4096 spheres, <= 8 bounces, 8 x 8 tile queues
    W, H = 1920, 1080
    sc = synth.sphere_scene(4096, seed=0)
    sc["scale"] = synth.camera_scale(W, H)
    props = torch.cuda.get_device_properties(dev)
    for k in kinds:
        r = gq.Renderer(k, sc, W, H, tiles=(8, 8), max_bounces=8)
        r.render()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r.render()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = r.stats.cpu().numpy()
        assert st[2] == 0 and st[1] == W * H
        t = float(np.median(ms))
        segs = int(st[0])
        # ALU roofline: 17 fp32 operations per ray-sphere test (no fused multiply-add),
        # one test per sphere per segment; peak = SMs x 128 fp32 lanes x max SM clock
        flops = segs * 4096 * 17
        peak = props.multi_processor_count * 128 * 2.07e9
        out["rt_1920x1080_%s" % k] = {"ms": round(t, 3), "segments": segs, "mrays_s": round(segs / (t * 1e-3) / 1e6, 1),
                                      "alu_tops": round(flops / (t * 1e-3) / 1e12, 2),
                                      "alu_frac_of_peak": round(flops / (t * 1e-3) / peak, 3)}
        for q in r.queues:
            q.close()
    return out


def _timed(fn, reps, spread=None):
    """Median device time (ms) of `reps` timed calls after an untimed one;
    `spread` (a list) receives (min, max)."""
    import torch
    fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    if spread is not None:
        spread[:] = [min(ms), max(ms)]
    return float(np.median(ms))


def bench_batched(gq, synth, kinds, dev, reps=7):
    """Batched forms against the plain per-call form on the same GPU.
    (1) 256 independent queues, capacities log-uniform 2^8 .. 2^16 (seed 0),
        2^18 threads (1024 per queue), 10^7 operations, 50 % producers; one step
        resets every queue and runs the workload: per-call = 256 launches,
        persistent = one launch, graph = the step captured and replayed,
        tuned = autotuned batch width / blocks / back-off, graph-replayed.
    (2) 64 BFS instances, R-MAT scale uniform in 12 .. 18 (seed 11): per-call =
        one gq_bfs per instance, batched = one persistent launch (8-block clusters)."""
    import torch
    from paper_2606_01693_gb300 import autotune
    out = {}
    Q, TPQ, OPS = 256, 1024, 10 ** 7
    OPQ, PPQ = OPS // Q, TPQ // 2
    r = synth.splitmix64(0, np.arange(Q)) >> np.uint64(40)
    caps = 1 << (8 + (r.astype(np.float64) * 2.0**-24 * 9).astype(np.int64))
    for k in kinds:
        qc = caps if k != "ymc" else np.full(Q, 3 * OPQ + (1 << 12))
        mq = gq.MultiQueue(k, qc, 8, TPQ)
        counts = torch.zeros(8, dtype=torch.int64, device=dev)

        def succ():
            c = counts.cpu().numpy()
            return float(c[0] + c[2])

        def per_call():
            counts.zero_()
            for q in mq.queues:
                q.reset()
            mq.run_per_call(TPQ, PPQ, OPQ, counts)

        def persistent():
            counts.zero_()
            mq.reset()
            mq.run(TPQ, PPQ, OPQ, counts)

        res = {}

        def mops(name, fn):
            sp = []
            t = _timed(fn, reps, sp)
            ok = succ()
            res[name + "_mops"] = round(ok / (t * 1e-3) / 1e6, 1)
            # Mops/s of the slowest and the fastest repetition (the last one's operation count)
            res[name + "_mops_range"] = [round(ok / (sp[1] * 1e-3) / 1e6, 1), round(ok / (sp[0] * 1e-3) / 1e6, 1)]

        mops("per_call", per_call)
        mops("persistent", persistent)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            persistent()
        mops("graph", g.replay)
        best = autotune.tune_multi(mq, TPQ, PPQ, OPQ, widths=(32, 16, 8), blocks_per_sm=(0, 4), backoffs=(0, 200),
                                   reps=3)
        g2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g2):
            counts.zero_()
            mq.reset()
            mq.run(TPQ, PPQ, OPQ, counts, blocks=best["blocks"])
        mops("tuned_graph", g2.replay)
        res["tuned"] = {kk: best[kk] for kk in ("batch_width", "blocks", "backoff_ns", "patience", "help_delay")}
        out["queues256_%s" % k] = res
        mq.close()
    # batched BFS
    rr = synth.splitmix64(11, np.arange(64)) >> np.uint64(40)
    scales = 12 + (rr.astype(np.float64) * 2.0**-24 * 7).astype(np.int64)
    graphs = [synth.rmat_csr_fast(int(sc), seed=11000 + i) for i, sc in enumerate(scales)]
    sources = [0] * len(graphs)
    for k in kinds:
        b = gq.BatchBfs(k, graphs, sources, slots=64, cluster_blocks=8)
        t_b = _timed(b.run, reps)
        nmax = max(len(o) - 1 for o, _ in graphs)
        cap = 3 * nmax + 64 * 65 + (1 << 16) if k == "ymc" else min(1 << max(12, (nmax - 1).bit_length()), 1 << 23)
        qa, qb = gq.Queue(k, cap, 4, 1 << 19), gq.Queue(k, cap, 4, 1 << 19)
        st = torch.zeros(4, dtype=torch.int64, device=dev)

        def per_call_bfs():
            for (d_off, d_adj, dist) in b.graphs:
                qa.reset()
                qb.reset()
                gq.gq_bfs(qa.handle, qb.handle, d_off, d_adj, 0, dist, st)

        t_p = _timed(per_call_bfs, reps)
        out["bfs64_%s" % k] = {"per_call_ms": round(t_p, 2), "batched_ms": round(t_b, 2),
                               "speedup": round(t_p / t_b, 2)}
        qa.close()
        qb.close()
    return out


def bench_serving(gq, synth, kinds, dev, pool_graphs=1000, seed=2026):
    """BFS serving: a resident pool of R-MAT graphs (scale uniform in 10..20 by
    seed, i.e. log-uniform vertex counts), requests (graph, source) with Poisson
    arrivals at 100..10,000 req/s, admission against a 32 GiB budget.  Persistent
    device scheduler (clusters of 8 blocks fed by the mapped request ring) vs one
    gq_bfs launch per request vs the adaptive mode that switches between the two;
    the persistent scheduler with its default gangs (up to 16 clusters for a
    request on a graph of at least 2^17 vertices) and without (`_solo`).
    Latency = host-observed completion - arrival."""
    import torch
    scales = synth.rmat_pool_scales(pool_graphs, 10, 20, seed)
    t0 = time.perf_counter()
    # the pool is generated on the device (same graphs as the host generator)
    devg = [synth.rmat_csr_torch(int(sc), seed=seed * 1000 + i, device=dev) for i, sc in enumerate(scales)]
    offs = [o.cpu().numpy().view(np.uint64) for o, _ in devg]
    gen_s = time.perf_counter() - t0
    out = {"pool": {"graphs": pool_graphs, "scales": "uniform 10..20", "edges": int(sum(a.numel() for _, a in devg)),
                    "device_gib": round(sum(o.numel() * 8 + a.numel() * 4 for o, a in devg) / 2**30, 2),
                    "generated_s": round(gen_s, 1), "budget_gib": 32}}
    for rate in (100, 300, 1000, 3000, 10000):
        nreq = int(min(2000, max(200, rate)))
        gid, src, arr = synth.serving_requests(offs, nreq, float(rate), seed + rate)
        for k in kinds:
            for mode in ("persistent", "persistent_solo", "per_request", "adaptive"):
                # persistent_solo: the scheduler without gangs (one cluster per request)
                r = gq.gq_serve(k, devg, gid, src, arr, mode=mode.replace("_solo", ""), cluster_blocks=8,
                                budget_bytes=32 << 30, gang_clusters=1 if mode.endswith("_solo") else 0)
                lat = r["latency_s"] * 1e3
                out["%s_%s_%d" % (k, mode, rate)] = {
                    "requests": nreq, "p50_ms": round(float(np.percentile(lat, 50)), 3),
                    "p99_ms": round(float(np.percentile(lat, 99)), 3),
                    "throughput_rps": round(nreq / r["wall_s"], 1), "admission_waits": int(r["admission_waits"]),
                    "peak_state_gib": round(r["peak_state_bytes"] / 2**30, 3), "slots": int(r["slots_used"]),
                    "persistent_requests": int(r["persistent_requests"]), "gang_requests": int(r["gang_requests"])}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import synth
    T, K = args.threads, args.ops
    # every step a bounded sample: the --cpu-threads budget shared by all steps
    # (warm-up included), so the whole run takes about as long as one CPU baseline
    per_step = max(1 << 12, args.cpu_threads // max(1, args.steps + args.warmup))
    Ts = min(T, 1 << (per_step.bit_length() - 1))
    sched = synth.mixed_schedule_bits(args.seed, Ts, K)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.mutex_run(1, Ts, K, sched=sched, nthreads=cores)
    tot_s, tot_ops = 0.0, 0
    for _ in range(args.steps):
        secs, c, nt = oracle.mutex_run(1, Ts, K, sched=sched, nthreads=cores)
        tot_s += secs
        tot_ops += int(c[0] + c[2])
    v = tot_ops / tot_s / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mops/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": workload_config(args, args.kinds.split(",") if args.kinds else ALL_KINDS, world),
            "cpu_baseline": {"value": v, "unit": "Mops/s", "cores": cores, "kind": "oracle",
                             "sample": "the oracle's mutex-guarded std::deque (unbounded) on the first %d of %d "
                                       "logical threads x %d ops of the same schedule, per step" % (Ts, T, K)},
            "e2e": {"value": v, "unit": "Mops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import paper_2606_01693_gb300 as gq
    import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    T, K = args.threads, args.ops
    kinds = args.kinds.split(",") if args.kinds else list(gq.READY_KINDS)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- same-box atomic peaks (roofline denominators) ----
    peak_buf = torch.zeros(1 << 21, dtype=torch.int64, device=dev)     # 16 MiB, L2-resident
    sink = torch.zeros(1, dtype=torch.int64, device=dev)

    def time_peak(pattern, iters, reps=4):
        # a peak: the best of `reps` timed launches after one untimed launch
        blocks, threads = sms * 8, 256
        gq.gq_atomic_peak(pattern, blocks, threads, iters, peak_buf, sink)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gq.gq_atomic_peak(pattern, blocks, threads, iters, peak_buf, sink)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        ops = blocks * threads * iters
        if pattern in (gq.GQ_PEAK_SAME_ADDR_FAA, gq.GQ_PEAK_SPREAD_FAA, gq.GQ_PEAK_PACKED_FAA):
            ops //= 32
        return ops / (best * 1e-3) / 1e9

    peaks = {"same_addr_faa_gops": time_peak(gq.GQ_PEAK_SAME_ADDR_FAA, 256),
             "coalesced_cas_gops": time_peak(gq.GQ_PEAK_COALESCED_CAS, 256),
             "scattered_cas_gops": time_peak(gq.GQ_PEAK_SCATTERED_CAS, 256),
             "coalesced_load_gops": time_peak(gq.GQ_PEAK_COALESCED_LOAD, 256),
             "faa_16_counters_4k_apart_gops": time_peak(gq.GQ_PEAK_SPREAD_FAA, 256),
             "faa_16_counters_128b_apart_gops": time_peak(gq.GQ_PEAK_PACKED_FAA, 256)}

    # ---- workload ----
    sched = synth.mixed_schedule_bits(args.seed, T, K)
    dsched = torch.from_numpy(sched.view(np.int64)).to(dev)
    # G-WFQ-YMC never reuses cells: its pool covers every ticket of a step
    # (about one per operation, plus tickets burned by races), here 1.25x the
    # operations plus 2^21 for the batch-API leg.
    ymc_pool = int(1.25 * T * K) + (1 << 21)
    queues = {k: gq.Queue(k, CAPACITY if k != "ymc" else ymc_pool, 8, max_threads=T) for k in kinds}
    counts = {k: torch.zeros(8, dtype=torch.int64, device=dev) for k in kinds}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    launches_per_step = {"lfq": 3, "wfq": 3, "ymc": 2}

    def step(evs=None):
        for k in kinds:
            queues[k].reset()
            if evs is not None:
                evs[k][0].record()
            gq.gq_run(queues[k].handle, gq.GQ_RUN_MIXED, T, block=256, ops=K, sched=dsched, counts=counts[k])
            if evs is not None:
                evs[k][1].record()

    clk = Clocks(local)                      # started before the warm-up: sampling by the timed region
    for _ in range(args.warmup):
        step()
    for k in kinds:
        st = queues[k].sync_status()
        if st != 0:
            raise SystemExit("device error in warm-up: %s" % gq.status_str(st))
        counts[k].zero_()
    barrier()
    t_region = time.time()
    step_ms, kern_ms = [], {k: 0.0 for k in kinds}
    for _ in range(args.steps):
        flush.fill_(1)                       # L2 flush between timed steps (256 MiB write)
        evs = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for k in kinds}
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        step(evs)
        s1.record()
        s1.synchronize()
        step_ms.append(s0.elapsed_time(s1))
        for k in kinds:
            kern_ms[k] += evs[k][0].elapsed_time(evs[k][1])
    barrier()
    clocks = clk.stop(window=(t_region, time.time()))
    for k in kinds:
        st = queues[k].sync_status()
        if st != 0:
            raise SystemExit("device error: %s" % gq.status_str(st))
    c = {k: counts[k].cpu().numpy().view(np.uint64) for k in kinds}
    succ = {k: int(c[k][gq.GQ_CNT_ENQ_OK] + c[k][gq.GQ_CNT_DEQ_OK]) for k in kinds}
    for k in kinds:
        assert c[k][gq.GQ_CNT_ERRORS] == 0, k
    total_ms, all_succ = replica_totals(float(sum(step_ms)), sum(succ.values()), dev)
    value = all_succ / (total_ms * 1e-3) / 1e6

    # ---- roofline of the dominant run kernel ----
    # Section III: a successful ring operation (G-LFQ, G-WFQ) is two slot RMWs
    # (one per index ring) and 2/W counter fetch-and-adds; a G-WFQ-YMC one is one
    # cell RMW (the value CAS, or the dequeue's claim) and 1/W fetch-and-add.
    # Two ceilings bound the rate: the slots' (coalesced-CAS rate / slot RMWs per
    # op) and the hot counters' (each counter serves W tickets per fetch-and-add
    # at the single-address rate; a balanced run spreads its operations over two
    # counters per direction, 2 W P_single).  The binding one is the smaller.
    W = 32
    per_queue = {}
    for k in kinds:
        t_s = kern_ms[k] * 1e-3
        ops_s = succ[k] / t_s
        slot_rmw = 1.0 if k == "ymc" else 2.0
        ctr_per_op = (1.0 if k == "ymc" else 2.0) / W
        atom_rate = ops_s * (slot_rmw + ctr_per_op)
        slot_ceiling = peaks["coalesced_cas_gops"] * 1e9 / slot_rmw
        counter_ceiling = 2 * W * peaks["same_addr_faa_gops"] * 1e9
        ceiling = min(slot_ceiling, counter_ceiling)
        per_queue[k] = {"kernel_mops": ops_s / 1e6, "kernel_ms_per_launch": kern_ms[k] / args.steps,
                        "succ_ops_per_launch": succ[k] // args.steps,
                        "algorithmic_atomics_per_succ_op": slot_rmw + ctr_per_op,
                        "achieved_gatomic_s": atom_rate / 1e9,
                        "slot_ceiling_mops": slot_ceiling / 1e6, "counter_ceiling_mops": counter_ceiling / 1e6,
                        "binding": "counter" if counter_ceiling < slot_ceiling else "slot",
                        "frac_of_binding_ceiling": ops_s / ceiling,
                        "empty": int(c[k][gq.GQ_CNT_DEQ_EMPTY]) // args.steps,
                        "full": int(c[k][gq.GQ_CNT_ENQ_FULL]) // args.steps}
    # measured fast-path events per successful operation: one launch of the
    # counting instantiation on the same workload (never timed)
    for k in kinds:
        oc = torch.zeros(gq.GQ_OC_N, dtype=torch.int64, device=dev)
        cc = torch.zeros(8, dtype=torch.int64, device=dev)
        queues[k].reset()
        gq.gq_run(queues[k].handle, gq.GQ_RUN_MIXED, T, block=256, ops=K, sched=dsched, counts=cc, opcount=oc)
        torch.cuda.synchronize()
        cn = cc.cpu().numpy()
        s_ok = float(cn[gq.GQ_CNT_ENQ_OK] + cn[gq.GQ_CNT_DEQ_OK])
        o = dict(zip(gq.OC_NAMES, oc.cpu().numpy().tolist()))
        atomics = o["faa"] + o["cas"] + o["rmw"] + o["threshold"] + o["catchup"]
        per_queue[k]["measured"] = {"atomics_per_succ_op": round(atomics / s_ok, 4),
                                    "per_succ_op": {nm: round(v / s_ok, 4) for nm, v in o.items()},
                                    "cas_fail_frac": round(o["cas_fail"] / max(1, o["cas"]), 4)}
    dom = max(kinds, key=lambda k: kern_ms[k])
    pq = per_queue[dom]
    traffic = NCU_TRAFFIC.get(dom)
    bind = min(pq["slot_ceiling_mops"], pq["counter_ceiling_mops"])
    roofline = {"bound": "l2_atomic", "kernel": "k_run<u64,%s> (mixed 50/50)" % dom.upper(),
                "achieved": pq["kernel_mops"] / 1e3, "peak": bind / 1e3, "unit": "G succ ops/s",
                "frac": pq["frac_of_binding_ceiling"], "traffic": traffic,
                "binding": pq["binding"],
                "slot_ceiling": pq["slot_ceiling_mops"] / 1e3, "counter_ceiling": pq["counter_ceiling_mops"] / 1e3,
                "achieved_gatomic_s": pq["achieved_gatomic_s"],
                "frac_of_coalesced_cas": pq["achieved_gatomic_s"] / peaks["coalesced_cas_gops"],
                "peak_source": "measured live on this GPU: min(coalesced 64-bit CAS rate / slot RMWs per op, "
                               "2 x 32 x same-address fetch-add rate)"}

    # ---- imbalanced producer / consumer split (capacity 2^16, 2^18 threads, 10^7 ops) ----
    split = {}
    if not args.no_sweep:
        Ts, total, cap = 1 << 18, 10 ** 7, 1 << 16
        for k in kinds:
            qs = gq.Queue(k, cap if k != "ymc" else int(1.4 * total), 8, max_threads=Ts)
            for frac in (0.1, 0.5, 0.9):
                P = int(frac * Ts)
                cc = torch.zeros(8, dtype=torch.int64, device=dev)
                best = None
                for rep in range(3):
                    qs.reset()
                    cc.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    gq.gq_run(qs.handle, gq.GQ_RUN_SPLIT, Ts, producers=P, total_ops=total, counts=cc)
                    e1.record()
                    e1.synchronize()
                    ms = e0.elapsed_time(e1)
                    if rep and (best is None or ms < best[0]):
                        best = (ms, cc.cpu().numpy().copy())
                st = qs.sync_status()
                assert st == 0, (k, frac, gq.status_str(st))
                ms, cn = best
                ok = float(cn[gq.GQ_CNT_ENQ_OK] + cn[gq.GQ_CNT_DEQ_OK])
                pqk = per_queue[k]
                ceiling = min(pqk["slot_ceiling_mops"], pqk["counter_ceiling_mops"]) * 1e6
                # one direction only is busy on its counters when the split is lopsided; the
                # balanced ceiling is the reference either way
                split["%s_p%d" % (k, int(frac * 100))] = {
                    "succ_mops": round(ok / (ms * 1e-3) / 1e6, 1),
                    "attempted_mops": round(total / (ms * 1e-3) / 1e6, 1), "ms": round(ms, 3),
                    "enq_ok": int(cn[gq.GQ_CNT_ENQ_OK]), "full": int(cn[gq.GQ_CNT_ENQ_FULL]),
                    "deq_ok": int(cn[gq.GQ_CNT_DEQ_OK]), "empty": int(cn[gq.GQ_CNT_DEQ_EMPTY]),
                    "frac_of_binding_ceiling": round(ok / (ms * 1e-3) / ceiling, 4)}
            qs.close()

    # ---- sweep over thread counts (kernel only, untimed region) ----
    sweep = {}
    if not args.no_sweep:
        for k in kinds:
            sweep[k] = {}
            for lg in range(10, 21):
                Ts = 1 << lg
                if Ts > T:
                    break
                sb = torch.from_numpy(synth.mixed_schedule_bits(args.seed, Ts, K).view(np.int64)).to(dev)
                cc = torch.zeros(8, dtype=torch.int64, device=dev)
                queues[k].reset()
                gq.gq_run(queues[k].handle, gq.GQ_RUN_MIXED, Ts, ops=K, sched=sb, counts=cc)
                queues[k].reset()
                cc.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                gq.gq_run(queues[k].handle, gq.GQ_RUN_MIXED, Ts, ops=K, sched=sb, counts=cc)
                e1.record()
                e1.synchronize()
                cn = cc.cpu().numpy()
                sweep[k][str(Ts)] = round((cn[0] + cn[2]) / (e0.elapsed_time(e1) * 1e-3) / 1e6, 1)

    # ---- enqueue-only then dequeue-only phases (kernel only, untimed region) ----
    # every thread enqueues its share of min(2^20, T * ops) items, then (second
    # launch) every thread dequeues the same number
    phases = {}
    if not args.no_sweep:
        for k in kinds:
            phases[k] = {}
            for Ts in [1 << lg for lg in range(10, 21) if (1 << lg) <= T]:
                target = min(CAPACITY, Ts * K)
                cc = torch.zeros(8, dtype=torch.int64, device=dev)
                res = {}
                for rep in range(2):
                    queues[k].reset()
                    cc.zero_()
                    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                    ev[0].record()
                    gq.gq_run(queues[k].handle, gq.GQ_RUN_SPLIT, Ts, producers=Ts, total_ops=target, counts=cc)
                    ev[1].record()
                    gq.gq_run(queues[k].handle, gq.GQ_RUN_SPLIT, Ts, producers=0, total_ops=target, counts=cc)
                    ev[2].record()
                    ev[2].synchronize()
                    cn = cc.cpu().numpy()
                    assert cn[gq.GQ_CNT_ENQ_OK] == target and cn[gq.GQ_CNT_DEQ_OK] == target, (k, Ts, cn)
                    res = {"items": target,
                           "enqueue_mops": round(target / (ev[0].elapsed_time(ev[1]) * 1e-3) / 1e6, 1),
                           "dequeue_mops": round(target / (ev[1].elapsed_time(ev[2]) * 1e-3) / 1e6, 1)}
                phases[k][str(Ts)] = res

    # ---- end to end through the public batch API with host buffers ----
    # One step: for every queue kind, pinned host -> device copy of 2^20 items,
    # gq_enqueue_batch, gq_dequeue_batch, device -> host copy of the values and
    # the counts.  Each kind runs on its own stream, so one kind's copies
    # overlap another's kernels; the host reads every step's counts, one step
    # behind the launches.
    e2e = None
    if not args.no_e2e:
        n = CAPACITY
        # queues of their own, sized for the batch (G-WFQ-YMC: a pool of 3 x 2^20 cells for the batch's 2^21
        # tickets, not the headline's 1.3 x 10^8, whose reset alone would clear 3 GB per step); the batch
        # kernels run at most one resident wave of threads and never more threads than records: 2^17
        # records (the enqueue and dequeue rates peak at 2^17 - 2^18 threads, `phases`) keep each reset's
        # record clear at 2 x 16 MiB for G-WFQ instead of 2 x 128 MiB
        eq = {k: gq.Queue(k, CAPACITY if k != "ymc" else 3 * CAPACITY, 8, max_threads=E2E_THREADS)
              for k in kinds}
        streams = {k: torch.cuda.Stream(device=dev) for k in kinds}
        host_items = torch.arange(1, n + 1, dtype=torch.int64).pin_memory()
        # two sets of host result buffers: step s + 1 is launched before the
        # host waits for step s's counts, so its copies must not land where
        # the host is still reading
        bufs = {k: {"out": [torch.empty(n, dtype=torch.int64).pin_memory() for _ in range(2)],
                    "cnt": [torch.empty(2, dtype=torch.int64).pin_memory() for _ in range(2)],
                    "done": [torch.cuda.Event() for _ in range(2)],
                    "d_items": torch.empty(n, dtype=torch.int64, device=dev),
                    "d_out": torch.empty(n, dtype=torch.int64, device=dev),
                    "d_cnt": torch.zeros(2, dtype=torch.int64, device=dev)} for k in kinds}
        torch.cuda.synchronize()

        def e2e_launch(s):
            par = s & 1
            for k in kinds:
                b = bufs[k]
                with torch.cuda.stream(streams[k]):
                    eq[k].reset()
                    b["d_items"].copy_(host_items, non_blocking=True)
                    gq.gq_enqueue_batch(eq[k].handle, b["d_items"], n, None, b["d_cnt"][0:1])
                    gq.gq_dequeue_batch(eq[k].handle, b["d_out"], n, None, b["d_cnt"][1:2])
                    b["out"][par].copy_(b["d_out"], non_blocking=True)
                    b["cnt"][par].copy_(b["d_cnt"], non_blocking=True)
                    b["done"][par].record(streams[k])

        def e2e_collect(s):
            par = s & 1
            tot = 0
            for k in kinds:
                bufs[k]["done"][par].synchronize()
                tot += int(bufs[k]["cnt"][par][0]) + int(bufs[k]["cnt"][par][1])
            return tot

        for w in range(3):
            e2e_launch(w)
            assert e2e_collect(w) == 2 * n * len(kinds)
        t0 = time.perf_counter()
        tot = 0
        e2e_launch(0)
        for st in range(args.steps):
            if st + 1 < args.steps:
                e2e_launch(st + 1)
            tot += e2e_collect(st)
        dt = time.perf_counter() - t0
        for k in kinds:
            assert eq[k].sync_status() == 0
            eq[k].close()
        e2e = {"value": tot / dt / 1e6, "unit": "Mops/s", "h2d_bytes_per_step": 8 * n * len(kinds),
               "d2h_bytes_per_step": (8 * n + 16) * len(kinds),
               "how": "per queue kind on its own stream: reset, pinned H2D of 2^20 items, gq_enqueue_batch, "
                      "gq_dequeue_batch, D2H of values and counts; the kinds' streams overlap, and step s + 1 is "
                      "launched before the host waits for and reads step s's counts (two sets of host result "
                      "buffers); wall clock over %d steps" % args.steps}

    apps = None
    if not args.no_apps:
        apps = bench_apps(gq, synth, kinds, dev)
    batched = None
    if not args.no_batched:
        batched = bench_batched(gq, synth, kinds, dev)
    serving = None
    if not args.no_serving and rank == 0:
        serving = bench_serving(gq, synth, kinds, dev)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(T, K, args.seed, args.cpu_threads)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Mops/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": workload_config(args, kinds, world),
                "roofline": roofline, "peaks": peaks, "per_queue": per_queue, "sweep": sweep, "phases": phases,
                "split_2p18_cap2p16": split,
                "cpu_baseline": cpu, "e2e": e2e, "apps": apps, "batched": batched, "serving": serving,
                "gpu_launches": args.steps * sum(launches_per_step[k] for k in kinds),
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
