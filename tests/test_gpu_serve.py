"""Serving on the GPU (run with -m gpu): BFS requests served by the persistent
device scheduler (host request ring in mapped pinned memory) and by one launch
per request.  Every request's distances must equal the oracle's sequential
BFS, and be the same whether the request is served alone or in the mix."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_01693_gb300 as gq
import synth

pytestmark = pytest.mark.gpu
KINDS = list(gq.READY_KINDS)
MODES = ["persistent", "per_request", "adaptive"]


@pytest.fixture(scope="module")
def pool():
    host = [synth.rmat_csr_fast(int(s), seed=900 + i) for i, s in enumerate([6, 8, 9, 10, 11, 12])]
    host.append(synth.grid_csr(48, 20))      # a deep graph: 66 levels
    dev = [(torch.from_numpy(o.view(np.int64)).cuda(), torch.from_numpy(a.view(np.int32)).cuda()) for o, a in host]
    return host, dev


def _expected(host, gid, src):
    memo = {}
    out = []
    for g, s in zip(gid, src):
        key = (int(g), int(s))
        if key not in memo:
            memo[key] = oracle.bfs(host[g][0], host[g][1], int(s))
        out.append(memo[key])
    return out


def _outs(host, gid):
    return [torch.empty(len(host[g][0]) - 1, dtype=torch.int32, device="cuda") for g in gid]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mode", MODES)
def test_mix_matches_cpu_bfs(pool, kind, mode):
    host, dev = pool
    gid, src, arr = synth.serving_requests([h[0] for h in host], 48, 4000.0, seed=21)
    outs = _outs(host, gid)
    r = gq.gq_serve(kind, dev, gid, src, arr, mode=mode, slots=6, cluster_blocks=2, outs=outs)
    torch.cuda.synchronize()
    assert (r["latency_s"] >= 0).all()
    assert r["wall_s"] >= r["latency_s"][-1] - 1e-9
    want = _expected(host, gid, src)
    for o, w in zip(outs, want):
        assert (o.cpu().numpy().view(np.uint32) == w).all()
    if mode == "persistent":
        assert r["slots_used"] == 6
        reached_edges = sum(int(np.diff(host[g][0].astype(np.int64))[w != 0xFFFFFFFF].sum())
                            for g, w in zip(gid, want))
        assert r["edges_scanned"] == reached_edges


@pytest.mark.parametrize("kind", KINDS)
def test_sixteen_block_clusters(pool, kind):
    """Clusters above the portable size (16 blocks of 256 threads) serve the same distances."""
    host, dev = pool
    gid, src, arr = synth.serving_requests([h[0] for h in host], 16, 5000.0, seed=44)
    outs = _outs(host, gid)
    r = gq.gq_serve(kind, dev, gid, src, arr, mode="persistent", slots=4, cluster_blocks=16, outs=outs)
    assert r["slots_used"] >= 1 and (r["latency_s"] >= 0).all()
    for o, w in zip(outs, _expected(host, gid, src)):
        assert (o.cpu().numpy().view(np.uint32) == w).all()


@pytest.mark.parametrize("kind", KINDS)
def test_alone_equals_in_mix(pool, kind):
    """Each request served alone gives the bytes it gave in the mix (both modes)."""
    host, dev = pool
    gid, src, arr = synth.serving_requests([h[0] for h in host], 24, 20000.0, seed=33)
    mix = {}
    for mode in MODES:
        outs = _outs(host, gid)
        gq.gq_serve(kind, dev, gid, src, arr, mode=mode, slots=8, cluster_blocks=4, outs=outs)
        mix[mode] = [o.cpu().numpy() for o in outs]
    for i in range(0, 24, 3):
        o = _outs(host, gid[i:i + 1])
        gq.gq_serve(kind, dev, gid[i:i + 1], src[i:i + 1], [0.0], mode="persistent", slots=1, cluster_blocks=1,
                    outs=o)
        alone = o[0].cpu().numpy()
        assert (alone == mix["persistent"][i]).all()
        assert (alone == mix["per_request"][i]).all()


@pytest.mark.parametrize("mode", MODES)
def test_admission_waits_under_small_budget(pool, mode):
    """With room for about two requests' state, later requests wait; results stay exact."""
    host, dev = pool
    gid, src, arr = synth.serving_requests([h[0] for h in host], 40, 1e6, seed=5)   # a burst
    def charge(g):
        n, m = len(host[g][0]) - 1, int(host[g][0][-1])
        qb = gq.gq_workspace_bytes(gq.GQ_LFQ, max(4096, 1 << (n - 1).bit_length()), 4,
                                   512 if mode == "persistent" else 1 << 19)
        return 8 * (n + 1) + 4 * m + (4 * n + 255) // 256 * 256 + 2 * qb
    budget = int(2.2 * max(charge(int(g)) for g in set(gid.tolist())))
    r = gq.gq_serve("lfq", dev, gid, src, arr, mode=mode, slots=8, cluster_blocks=2, budget_bytes=budget)
    assert r["peak_state_bytes"] <= budget
    assert r["admission_waits"] > 0
    assert (r["latency_s"] >= 0).all()
    outs = _outs(host, gid)
    r = gq.gq_serve("lfq", dev, gid, src, arr, mode=mode, slots=8, cluster_blocks=2, budget_bytes=budget,
                    outs=outs)
    for o, w in zip(outs, _expected(host, gid, src)):
        assert (o.cpu().numpy().view(np.uint32) == w).all()


@pytest.mark.parametrize("kind", KINDS)
def test_adaptive_switches_both_ways(pool, kind):
    """A burst hands the requests to the persistent scheduler; after a quiet gap
    per-request launches serve the rest; every result equals the oracle's."""
    host, dev = pool
    g1, s1, a1 = synth.serving_requests([h[0] for h in host], 60, 1e6, seed=51)     # a burst at t ~ 0
    g2, s2, a2 = synth.serving_requests([h[0] for h in host], 6, 20.0, seed=52)     # sparse, after 0.25 s
    gid, src = np.concatenate([g1, g2]), np.concatenate([s1, s2])
    arr = np.concatenate([a1, 0.25 + a2])
    outs = _outs(host, gid)
    r = gq.gq_serve(kind, dev, gid, src, arr, mode="adaptive", slots=4, cluster_blocks=2, outs=outs,
                    switch_backlog=2)
    assert (r["latency_s"] >= 0).all()
    assert 0 < r["persistent_requests"] < len(gid)          # both engines served requests
    for o, w in zip(outs, _expected(host, gid, src)):
        assert (o.cpu().numpy().view(np.uint32) == w).all()


def test_request_larger_than_budget_rejected(pool):
    host, dev = pool
    with pytest.raises(gq.GqError) as ei:
        gq.gq_serve("lfq", dev, [5], [0], [0.0], budget_bytes=1 << 16)
    assert ei.value.status == gq.GQ_ERR_INVALID


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("rate", [300.0, 6000.0])
def test_gangs_match_cpu_bfs(pool, kind, rate):
    """Gangs: every request asks for up to 4 clusters (gang_min_vertices 1).  At a low
    rate idle clusters join and gangs form; at a high rate most requests run on one
    cluster.  Distances equal the oracle's either way, and the edges scanned by all
    members add up to the reached edges."""
    host, dev = pool
    gid, src, arr = synth.serving_requests([h[0] for h in host], 40, rate, seed=31)
    outs = _outs(host, gid)
    r = gq.gq_serve(kind, dev, gid, src, arr, mode="persistent", slots=8, cluster_blocks=2, outs=outs,
                    gang_clusters=4, gang_min_vertices=1)
    assert (r["latency_s"] >= 0).all()
    want = _expected(host, gid, src)
    for o, w in zip(outs, want):
        assert (o.cpu().numpy().view(np.uint32) == w).all()
    reached_edges = sum(int(np.diff(host[g][0].astype(np.int64))[w != 0xFFFFFFFF].sum()) for g, w in zip(gid, want))
    assert r["edges_scanned"] == reached_edges
    assert r["persistent_requests"] == len(gid)
    if rate < 1000:
        assert r["gang_requests"] > 0, r


@pytest.mark.parametrize("kind", KINDS)
def test_gangs_on_large_graphs_only(kind):
    """Only requests on graphs of at least gang_min_vertices vertices form gangs; a
    scale-16 graph served by gangs of up to 8 eight-block clusters gives the oracle's
    distances."""
    host = [synth.rmat_csr_fast(8, seed=61), synth.rmat_csr_fast(16, seed=62)]
    dev = [(torch.from_numpy(o.view(np.int64)).cuda(), torch.from_numpy(a.view(np.int32)).cuda()) for o, a in host]
    gid = np.array([0, 1, 0, 1, 0, 1], dtype=np.uint32)
    src = np.array([0, 0, 5, 17, 9, 3], dtype=np.uint32)
    arr = np.arange(6) * 2e-3
    outs = _outs(host, gid)
    r = gq.gq_serve(kind, dev, gid, src, arr, mode="persistent", slots=16, cluster_blocks=8, outs=outs,
                    gang_clusters=8, gang_min_vertices=1 << 12)
    for i, o in enumerate(outs):
        assert (o.cpu().numpy().view(np.uint32) == oracle.bfs(host[gid[i]][0], host[gid[i]][1], int(src[i]))).all(), i
    assert 0 < r["gang_requests"] <= 3, r


def test_ring_wraps(pool):
    """More requests than ring entries (4096): entries are reused once their request is done."""
    host, dev = pool
    small = [host[0], host[1]]
    gid, src, arr = synth.serving_requests([h[0] for h in small], 5000, 2e5, seed=8)
    r = gq.gq_serve("lfq", [dev[0], dev[1]], gid, src, arr, mode="persistent", slots=16, cluster_blocks=1)
    assert (r["latency_s"] >= 0).all()
    want = _expected(small, gid, src)
    edges = sum(int(np.diff(small[g][0].astype(np.int64))[w != 0xFFFFFFFF].sum()) for g, w in zip(gid, want))
    assert r["edges_scanned"] == edges


def test_device_wait_limit_reports_timeout(pool):
    """A scheduler cluster whose next request arrives after the wait limit gives up
    (bounded %globaltimer wait) and the call returns GQ_ERR_TIMEOUT; the context stays usable."""
    host, dev = pool
    with pytest.raises(gq.GqError) as ei:
        gq.gq_serve("lfq", dev, [0, 1], [0, 0], [0.0, 3.0], mode="persistent", slots=2, cluster_blocks=1,
                    wait_limit_s=0.3)
    assert ei.value.status == gq.GQ_ERR_TIMEOUT
    r = gq.gq_serve("lfq", dev, [0], [0], [0.0], mode="persistent", slots=1, cluster_blocks=1)
    assert r["latency_s"][0] >= 0


@pytest.mark.parametrize("mode", ["persistent", "adaptive"])
def test_full_size_pool_sampled(mode):
    """The serving workload's shape: R-MAT graphs of scales 10..20 (both ends present),
    Poisson arrivals at 10,000 req/s, 8-block clusters, 32 GiB budget; the distances
    of a sample of requests (the largest graphs among them) equal the oracle's."""
    scales = np.concatenate([[10, 20], synth.rmat_pool_scales(10, 10, 20, 2026)])
    host = [synth.rmat_csr_fast(int(s), seed=7000 + i) for i, s in enumerate(scales)]
    dev = [(torch.from_numpy(o.view(np.int64)).cuda(), torch.from_numpy(a.view(np.int32)).cuda()) for o, a in host]
    gid, src, arr = synth.serving_requests([h[0] for h in host], 400, 10000.0, seed=99)
    order = np.argsort(-scales[gid], kind="stable")
    sample = set(order[:6].tolist()) | set(range(0, 400, 67))
    outs = [torch.empty(len(host[g][0]) - 1, dtype=torch.int32, device="cuda") if i in sample else None
            for i, g in enumerate(gid)]
    r = gq.gq_serve("lfq", dev, gid, src, arr, mode=mode, cluster_blocks=8, budget_bytes=32 << 30, outs=outs)
    assert (r["latency_s"] >= 0).all()
    for i in sorted(sample):
        want = oracle.bfs(host[gid[i]][0], host[gid[i]][1], int(src[i]))
        assert (outs[i].cpu().numpy().view(np.uint32) == want).all(), i


def test_device_generated_graphs_equal_host_graphs():
    for scale, seed in ((12, 5), (15, 2026007)):
        o1, a1 = synth.rmat_csr_fast(scale, seed=seed)
        o2, a2 = synth.rmat_csr_torch(scale, seed=seed, device="cuda")
        assert (o2.cpu().numpy() == o1.astype(np.int64)).all()
        assert (a2.cpu().numpy() == a1.view(np.int32)).all()


def test_thousand_graph_pool_wfq_at_3k_rps():
    """The serving workload at its stated size: a pool of 1000 R-MAT graphs of
    scales 10..20 (generated on the device), Poisson arrivals at 3000 req/s,
    G-WFQ in adaptive mode under the 32 GiB budget: every request completes,
    the admitted state never exceeds the budget, and a sample of requests (the
    largest graphs among them) has the oracle's distances."""
    scales = synth.rmat_pool_scales(1000, 10, 20, 2026)
    dev = [synth.rmat_csr_torch(int(s), seed=2026 * 1000 + i, device="cuda") for i, s in enumerate(scales)]
    offs = [o.cpu().numpy().view(np.uint64) for o, _ in dev]
    gid, src, arr = synth.serving_requests(offs, 600, 3000.0, seed=5)
    order = np.argsort(-scales[gid], kind="stable")
    sample = set(order[:3].tolist()) | set(range(0, 600, 150))
    outs = [torch.empty(len(offs[g]) - 1, dtype=torch.int32, device="cuda") if i in sample else None
            for i, g in enumerate(gid)]
    r = gq.gq_serve("wfq", dev, gid, src, arr, mode="adaptive", cluster_blocks=8, budget_bytes=32 << 30, outs=outs)
    assert (r["latency_s"] >= 0).all()
    assert r["peak_state_bytes"] <= 32 << 30
    for i in sorted(sample):
        g = gid[i]
        want = oracle.bfs(offs[g], dev[g][1].cpu().numpy().view(np.uint32), int(src[i]))
        assert (outs[i].cpu().numpy().view(np.uint32) == want).all(), i
