"""Command-line runs of the applications on synthetic inputs (one GPU).

    python -m paper_2606_01693_gb300.cli bfs --rmat 22 --kinds lfq,wfq,ymc
    python -m paper_2606_01693_gb300.cli bfs --grid 4096
    python -m paper_2606_01693_gb300.cli render --width 1920 --height 1080 --spheres 4096
    python -m paper_2606_01693_gb300.cli serve --graphs 64 --rate 1000 --requests 1000

Each prints one JSON object per queue kind (device time from CUDA events on the
launching stream, after one untimed run).  Inputs come from the repository's
seeded generators (`synth`), so run it from the repository root.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_bfs(args) -> None:
    import torch

    import synth
    from . import Queue, gq_bfs
    if args.grid:
        off, adj = synth.grid_csr(args.grid, args.grid)
        name, levels_hint = "grid%d" % args.grid, 2 * args.grid
    else:
        off, adj = synth.rmat_csr_fast(args.rmat, seed=args.seed)
        name, levels_hint = "rmat%d" % args.rmat, 64
    n = len(off) - 1
    d_off = torch.from_numpy(off.view(np.int64)).cuda()
    d_adj = torch.from_numpy(adj.view(np.int32)).cuda()
    dist = torch.empty(n, dtype=torch.int32, device="cuda")
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    for k in args.kinds.split(","):
        cap = 3 * n + 64 * (levels_hint + 1) + (1 << 16) if k == "ymc" else min(1 << max(12, (n - 1).bit_length()), 1 << 23)
        qa, qb = Queue(k, cap, 4, 1 << 19), Queue(k, cap, 4, 1 << 19)
        ms = []
        for rep in range(args.reps + 1):
            qa.reset()
            qb.reset()
            e0, e1 = _events()
            e0.record()
            gq_bfs(qa.handle, qb.handle, d_off, d_adj, args.source, dist, stats)
            e1.record()
            e1.synchronize()
            if rep:
                ms.append(e0.elapsed_time(e1))
        st = stats.cpu().numpy()
        status = qa.sync_status() or qb.sync_status() or int(st[3])
        t = float(np.median(ms)) if ms else float("nan")
        print(json.dumps({"app": "bfs", "graph": name, "kind": k, "ms": round(t, 3), "levels": int(st[0]),
                          "reached": int(st[1]), "edges_scanned": int(st[2]),
                          "gteps": round(float(st[2]) / (t * 1e-3) / 1e9, 3) if ms else None, "status": status}),
              flush=True)
        qa.close()
        qb.close()


def run_render(args) -> None:
    import synth
    from . import Renderer
    sc = synth.sphere_scene(args.spheres, seed=args.seed)
    sc["scale"] = synth.camera_scale(args.width, args.height)
    for k in args.kinds.split(","):
        r = Renderer(k, sc, args.width, args.height, tiles=(args.tiles, args.tiles), max_bounces=args.bounces)
        ms = []
        for rep in range(args.reps + 1):
            e0, e1 = _events()
            e0.record()
            r.render()
            e1.record()
            e1.synchronize()
            if rep:
                ms.append(e0.elapsed_time(e1))
        st = r.stats.cpu().numpy()
        t = float(np.median(ms)) if ms else float("nan")
        print(json.dumps({"app": "render", "kind": k, "ms": round(t, 3), "segments": int(st[0]),
                          "pixels": int(st[1]), "errflags": int(st[2]),
                          "mrays_s": round(int(st[0]) / (t * 1e-3) / 1e6, 1) if ms else None}), flush=True)


def run_serve(args) -> None:
    import torch

    import synth
    from . import gq_serve
    scales = synth.rmat_pool_scales(args.graphs, args.min_scale, args.max_scale, args.seed)
    host = [synth.rmat_csr_fast(int(sc), seed=args.seed * 1000 + i) for i, sc in enumerate(scales)]
    dev = [(torch.from_numpy(o.view(np.int64)).cuda(), torch.from_numpy(a.view(np.int32)).cuda()) for o, a in host]
    gid, src, arr = synth.serving_requests([h[0] for h in host], args.requests, args.rate, args.seed + 1)
    for k in args.kinds.split(","):
        for mode in args.modes.split(","):
            r = gq_serve(k, dev, gid, src, arr, mode=mode, cluster_blocks=args.cluster_blocks,
                         budget_bytes=int(args.budget_gib * 2**30))
            lat = r["latency_s"] * 1e3
            print(json.dumps({"app": "serve", "kind": k, "mode": mode, "rate": args.rate, "requests": args.requests,
                              "p50_ms": round(float(np.percentile(lat, 50)), 3),
                              "p99_ms": round(float(np.percentile(lat, 99)), 3),
                              "throughput_rps": round(args.requests / r["wall_s"], 1),
                              "admission_waits": int(r["admission_waits"]), "slots": int(r["slots_used"]),
                              "persistent_requests": int(r["persistent_requests"])}),
                  flush=True)


def main(argv=None) -> None:
    p = argparse.ArgumentParser(prog="python -m paper_2606_01693_gb300.cli")
    sub = p.add_subparsers(dest="cmd", required=True)
    b = sub.add_parser("bfs", help="level-synchronous BFS with two frontier queues")
    b.add_argument("--rmat", type=int, default=22, help="R-MAT scale (vertices 2^scale, edge factor 16)")
    b.add_argument("--grid", type=int, default=0, help="side of a 4-neighbour grid (overrides --rmat)")
    b.add_argument("--source", type=int, default=0)
    r = sub.add_parser("render", help="tile-queue wavefront ray tracing")
    r.add_argument("--width", type=int, default=1920)
    r.add_argument("--height", type=int, default=1080)
    r.add_argument("--spheres", type=int, default=4096)
    r.add_argument("--tiles", type=int, default=8)
    r.add_argument("--bounces", type=int, default=8)
    s = sub.add_parser("serve", help="BFS serving: persistent scheduler vs per-request launches")
    s.add_argument("--graphs", type=int, default=64)
    s.add_argument("--min-scale", type=int, default=10)
    s.add_argument("--max-scale", type=int, default=20)
    s.add_argument("--rate", type=float, default=1000.0)
    s.add_argument("--requests", type=int, default=1000)
    s.add_argument("--modes", default="persistent,per_request,adaptive")
    s.add_argument("--cluster-blocks", type=int, default=8)
    s.add_argument("--budget-gib", type=float, default=32.0)
    for q in (b, r, s):
        q.add_argument("--kinds", default="lfq,wfq,ymc")
        q.add_argument("--seed", type=int, default=0)
        q.add_argument("--reps", type=int, default=3)
    args = p.parse_args(argv)
    {"bfs": run_bfs, "render": run_render, "serve": run_serve}[args.cmd](args)


if __name__ == "__main__":
    main()
