"""Pins for the oracle's sequential BFS (CPU only): closed forms on grids and
paths, scipy's breadth-first shortest paths on random graphs, and the
Graph500-style validity properties on R-MAT graphs."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("w,h", [(1, 1), (5, 3), (64, 64), (97, 13)])
def test_grid_closed_form(w, h):
    off, adj = synth.grid_csr(w, h)
    d = oracle.bfs(off, adj, 0)
    r, c = np.divmod(np.arange(w * h), w)
    assert (d == (r + c)).all()


def test_path_and_isolated():
    # 0-1-2-3 path plus isolated vertex 4
    off = np.array([0, 1, 3, 5, 6, 6], np.uint64)
    adj = np.array([1, 0, 2, 1, 3, 2], np.uint32)
    d = oracle.bfs(off, adj, 0)
    assert d.tolist() == [0, 1, 2, 3, 0xFFFFFFFF]
    d = oracle.bfs(off, adj, 2)
    assert d.tolist() == [2, 1, 0, 1, 0xFFFFFFFF]


@pytest.mark.parametrize("seed", range(4))
def test_matches_scipy_unweighted_shortest_path(seed):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(seed)
    n = 300
    m = 700
    s = rng.integers(0, n, m); t = rng.integers(0, n, m)
    keep = s != t
    key = np.unique(np.concatenate([s[keep] * n + t[keep], t[keep] * n + s[keep]]))
    src, dst = key // n, key % n
    off = np.zeros(n + 1, np.uint64); np.cumsum(np.bincount(src, minlength=n), out=off[1:])
    A = sp.csr_matrix((np.ones(len(src)), (src, dst)), shape=(n, n))
    ref = csgraph.shortest_path(A, unweighted=True, indices=0)
    d = oracle.bfs(off, dst.astype(np.uint32), 0)
    want = np.where(np.isinf(ref), 0xFFFFFFFF, ref).astype(np.uint64)
    assert (d.astype(np.uint64) == want).all()


def test_rmat_graph500_properties():
    off, adj = synth.rmat_csr(10, seed=1)
    d = oracle.bfs(off, adj, 0).astype(np.int64)
    INF = 0xFFFFFFFF
    n = len(off) - 1
    src = np.repeat(np.arange(n), np.diff(off.astype(np.int64)))
    dst = adj.astype(np.int64)
    both = (d[src] != INF) & (d[dst] != INF)
    assert (np.abs(d[src][both] - d[dst][both]) <= 1).all()        # edges span <= 1 level
    assert ((d[src] == INF) == (d[dst] == INF)).all()              # reached set closed under edges
    reached = np.flatnonzero((d != INF) & (np.arange(n) != 0))
    has_parent = np.zeros(n, bool)
    ok = (d[src] != INF) & (d[dst] == d[src] + 1)
    has_parent[dst[ok]] = True
    assert has_parent[reached].all()                               # every reached v has a d-1 neighbour
