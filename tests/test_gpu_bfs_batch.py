"""Batched BFS on the GPU (run with -m gpu): many uneven R-MAT instances in one
persistent launch, one per thread-block cluster at a time; every instance's
distances must equal the oracle's sequential BFS."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_01693_gb300 as gq
import synth

pytestmark = pytest.mark.gpu
KINDS = list(gq.READY_KINDS)


def _instances(count, lo, hi, seed):
    r = synth.splitmix64(seed, np.arange(count)) >> np.uint64(40)
    scales = lo + (r.astype(np.float64) * 2.0**-24 * (hi - lo + 1)).astype(np.int64)
    graphs = [synth.rmat_csr_fast(int(s), seed=seed * 1000 + i) for i, s in enumerate(scales)]
    sources = [int(synth.bfs_sources(g[0], seed + i, 1)[-1]) for i, g in enumerate(graphs)]
    return graphs, sources


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("cluster_blocks,slots", [(1, 8), (4, 16), (8, 4)])
def test_batched_instances_match_cpu_bfs(kind, cluster_blocks, slots):
    graphs, sources = _instances(12, 6, 13, 7)
    b = gq.BatchBfs(kind, graphs, sources, slots=slots, cluster_blocks=cluster_blocks)
    b.run()
    torch.cuda.synchronize()
    for q in b.frontier + [b.idq]:
        assert q.sync_status() == 0
    st = b.stats.cpu().numpy()
    assert st[0] == len(graphs) and st[3] == 0
    edges = 0
    for (off, adj), src, d in zip(graphs, sources, b.dists()):
        want = oracle.bfs(off, adj, src)
        got = d.cpu().numpy().view(np.uint32)
        assert (got == want).all()
        edges += int(off[np.flatnonzero(want != 0xFFFFFFFF)].size)
    # run twice on the same queues: they were left empty (G-WFQ-YMC: cells cleared)
    b.run()
    torch.cuda.synchronize()
    for (off, adj), src, d in zip(graphs, sources, b.dists()):
        assert (d.cpu().numpy().view(np.uint32) == oracle.bfs(off, adj, src)).all()


def test_full_size_64_instances():
    graphs, sources = _instances(64, 12, 18, 11)
    for kind in KINDS:
        b = gq.BatchBfs(kind, graphs, sources, slots=64, cluster_blocks=8)
        b.run()
        torch.cuda.synchronize()
        assert b.stats.cpu().numpy()[0] == 64
        for (off, adj), src, d in list(zip(graphs, sources, b.dists()))[::7]:
            assert (d.cpu().numpy().view(np.uint32) == oracle.bfs(off, adj, src)).all()
