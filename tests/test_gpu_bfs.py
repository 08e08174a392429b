"""Frontier-queue BFS on the GPU against the oracle's sequential BFS (run with
-m gpu): distances must be bit-identical (they are unique; only parents could
differ).  Grids also have the closed form dist(r, c) = r + c from corner 0."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_01693_gb300 as gq
import synth

pytestmark = pytest.mark.gpu
DEV = "cuda"
KINDS = list(gq.READY_KINDS)


def _queues(kind, n, max_threads=1 << 19, levels_hint=64):
    # records for every resident thread (152 SMs x 2048 < 2^19)
    if kind == "ymc":
        cap = 3 * n + 64 * (levels_hint + 1) + (1 << 16)
    else:
        cap = 1 << max(1, (n - 1).bit_length())
        if kind == "wfq":
            # G-WFQ's cycle soundness R > D k / n + 6 needs n > 64 k / 2^19
            cap = min(max(cap, 1 << 12), 1 << 23)
    return gq.Queue(kind, cap, 4, max_threads), gq.Queue(kind, cap, 4, max_threads)


def _run(kind, off, adj, src, levels_hint=64):
    n = len(off) - 1
    qa, qb = _queues(kind, n, levels_hint=levels_hint)
    d_off = torch.from_numpy(off.view(np.int64)).to(DEV)
    d_adj = torch.from_numpy(adj.view(np.int32)).to(DEV)
    dist = torch.empty(n, dtype=torch.int32, device=DEV)
    stats = torch.zeros(4, dtype=torch.int64, device=DEV)
    gq.gq_bfs(qa.handle, qb.handle, d_off, d_adj, int(src), dist, stats)
    assert qa.sync_status() == 0 and qb.sync_status() == 0
    st = stats.cpu().numpy()
    assert st[3] == 0, "grid barrier timed out"
    return dist.cpu().numpy().view(np.uint32), st


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("w,h", [(1, 1), (7, 3), (64, 64), (300, 5)])
def test_grid_closed_form(kind, w, h):
    off, adj = synth.grid_csr(w, h)
    d, st = _run(kind, off, adj, 0, levels_hint=w + h)
    r, c = np.divmod(np.arange(w * h), w)
    assert (d == (r + c)).all()
    assert st[0] == w + h - 1 and st[1] == w * h and st[2] == len(adj)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("scale,seed", [(10, 0), (14, 1), (16, 2)])
def test_rmat_matches_cpu_bfs(kind, scale, seed):
    off, adj = synth.rmat_csr_fast(scale, seed=seed)
    for src in synth.bfs_sources(off, seed, 2):
        want = oracle.bfs(off, adj, src)
        got, st = _run(kind, off, adj, src)
        assert (got == want).all(), np.flatnonzero(got != want)[:10]
        assert st[1] == int((want != 0xFFFFFFFF).sum())


def test_disconnected_and_isolated_source():
    # two components; source isolated -> only itself reached
    off = np.array([0, 0, 1, 2], np.uint64)
    adj = np.array([2, 1], np.uint32)
    for kind in KINDS:
        d, st = _run(kind, off, adj, 0)
        assert d.tolist() == [0, 0xFFFFFFFF, 0xFFFFFFFF]
        d, st = _run(kind, off, adj, 1)
        assert d.tolist() == [0xFFFFFFFF, 0, 1]


@pytest.mark.parametrize("kind", KINDS)
def test_full_size_rmat22(kind):
    off, adj = synth.rmat_csr_fast(22, seed=0)
    want = oracle.bfs(off, adj, 0)
    got, st = _run(kind, off, adj, 0)
    assert (got == want).all()


@pytest.mark.parametrize("kind", KINDS)
def test_full_size_grid4096(kind):
    off, adj = synth.grid_csr(4096, 4096)
    got, st = _run(kind, off, adj, 0, levels_hint=8192)
    r, c = np.divmod(np.arange(4096 * 4096), 4096)
    assert (got == (r + c)).all()
    assert st[0] == 8191
