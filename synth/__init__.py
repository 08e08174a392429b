"""Seeded synthetic input generators shared by the tests, the benchmark and the oracle.

This module holds no queue arithmetic: it only produces inputs (operation
schedules, payload tokens, graphs, scenes).  Both the CUDA path and the CPU
oracle consume these arrays; neither side imports the other.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014, with
the 64-bit finaliser constants published by Vigna).  ``splitmix64(seed, k)`` is
the (k+1)-th output of a SplitMix64 stream whose state starts at ``seed``:
    state_k = seed + (k + 1) * 0x9E3779B97F4A7C15   (mod 2**64)
    z = state_k; z = (z ^ z>>30) * 0xBF58476D1CE4E5B9
    z = (z ^ z>>27) * 0x94D049BB133111EB;  out = z ^ z>>31
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, ctr) -> np.ndarray:
    """Vectorised SplitMix64: output number ``ctr`` (0-based) of the stream seeded with ``seed``."""
    ctr = np.asarray(ctr, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (ctr + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


# ---------------------------------------------------------------------------
# Queue workloads
# ---------------------------------------------------------------------------

def mixed_schedule_bits(seed: int, threads: int, ops_per_thread: int) -> np.ndarray:
    """50/50 interleaved enqueue/dequeue schedule, packed as uint64 words.

    Operation ``i`` of thread ``t`` has flat index ``j = t * ops_per_thread + i``;
    it is an enqueue iff bit ``j & 63`` of word ``j >> 6`` is 1.  Word ``w`` is
    ``splitmix64(seed, w)``.
    """
    nbits = threads * ops_per_thread
    nwords = (nbits + 63) // 64
    return splitmix64(seed, np.arange(nwords, dtype=np.uint64))


def schedule_is_enq(bits: np.ndarray, threads: int, ops_per_thread: int) -> np.ndarray:
    """Unpack ``mixed_schedule_bits`` into a bool array of shape (threads, ops_per_thread)."""
    nbits = threads * ops_per_thread
    b = np.unpackbits(bits.view(np.uint8), bitorder="little")[:nbits]
    return b.astype(bool).reshape(threads, ops_per_thread)


def token64(producer, seq):
    """64-bit payload token of the device-side FIFO conformance run: (producer << 32) | (seq + 1)."""
    return (np.asarray(producer, dtype=np.uint64) << np.uint64(32)) | (np.asarray(seq, dtype=np.uint64) + np.uint64(1))


def token32(producer, seq):
    """32-bit payload token of the one-block pairs workload: (producer << 16) | seq."""
    return (np.asarray(producer, dtype=np.uint32) << np.uint32(16)) | np.asarray(seq, dtype=np.uint32)


def split_ops_per_thread(total_ops: int, threads: int) -> np.ndarray:
    """Even split of ``total_ops`` over ``threads``: thread t gets floor(total/T), the first (total mod T) get one more."""
    base, rem = divmod(total_ops, threads)
    k = np.full(threads, base, dtype=np.int64)
    k[:rem] += 1
    return k


def random_op_list(seed: int, n_ops: int, p_enq: float = 0.5, value_bits: int = 64) -> tuple[np.ndarray, np.ndarray]:
    """A single-thread op list: kinds (1 = enqueue, 0 = dequeue) and enqueue values.

    Values are distinct draws masked to ``value_bits``; used by sequential tests.
    """
    r = splitmix64(seed, np.arange(2 * n_ops, dtype=np.uint64))
    thr = np.uint64(int(p_enq * 2**32))
    kinds = ((r[0::2] >> np.uint64(32)) < thr).astype(np.uint8)
    vals = r[1::2]
    if value_bits < 64:
        vals = vals & np.uint64((1 << value_bits) - 1)
    return kinds, vals


# ---------------------------------------------------------------------------
# Graphs (CSR, uint32 vertex ids, sorted neighbour lists)
# ---------------------------------------------------------------------------

def _csr_from_pairs(n: int, src: np.ndarray, dst: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    key = (src.astype(np.uint64) << np.uint64(32)) | dst.astype(np.uint64)
    key = np.unique(key)
    s = (key >> np.uint64(32)).astype(np.int64)
    d = (key & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    counts = np.bincount(s, minlength=n)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(counts, out=offsets[1:])
    return offsets, d


def grid_csr(width: int, height: int) -> tuple[np.ndarray, np.ndarray]:
    """4-neighbour 2-D grid; vertex id = row * width + col; neighbour lists in
    increasing id order (up, left, right, down)."""
    n = width * height
    v = np.arange(n, dtype=np.int64)
    r, c = v // width, v % width
    has = [r > 0, c > 0, c < width - 1, r < height - 1]
    nb = [v - width, v - 1, v + 1, v + width]
    deg = sum(h.astype(np.int64) for h in has)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(deg, out=offsets[1:])
    adj = np.empty(int(offsets[-1]), dtype=np.uint32)
    pos = offsets[:-1].astype(np.int64).copy()
    for h, w in zip(has, nb):
        adj[pos[h]] = w[h]
        pos[h] += 1
    return offsets, adj


_clib = None


def _lib():
    """Loads (building if needed) the C++ generator helpers in gen.cpp."""
    global _clib
    if _clib is None:
        import ctypes
        import os
        import subprocess
        here = os.path.dirname(os.path.abspath(__file__))
        so = os.path.join(here, "libsynth.so")
        srcf = os.path.join(here, "gen.cpp")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(srcf):
            tmp = so + ".tmp%d" % os.getpid()
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", tmp, srcf])
            os.replace(tmp, so)
        L = ctypes.CDLL(so)
        P, i64, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64
        L.synth_rmat_pairs.argtypes = [ctypes.c_int, i64, u64, u64, u64, u64, P, P]
        L.synth_rmat_pairs.restype = i64
        L.synth_csr.argtypes = [i64, i64, P, P, P, P]
        L.synth_csr.restype = i64
        _clib = L
    return _clib


def rmat_csr_fast(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
                  seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Same graph as rmat_csr, generated by the C++ helper (multi-threaded)."""
    L = _lib()
    n = 1 << scale
    m = edge_factor * n
    src = np.empty(2 * m, dtype=np.uint32)
    dst = np.empty(2 * m, dtype=np.uint32)
    k = L.synth_rmat_pairs(scale, m, seed & 0xFFFFFFFFFFFFFFFF, int(a * 2**32), int((a + b) * 2**32),
                           int((a + b + c) * 2**32), src.ctypes.data, dst.ctypes.data)
    offsets = np.empty(n + 1, dtype=np.uint64)
    adj = np.empty(k, dtype=np.uint32)
    e = L.synth_csr(n, k, src.ctypes.data, dst.ctypes.data, offsets.ctypes.data, adj.ctypes.data)
    return offsets, adj[:e].copy()


def rmat_csr(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
             seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """R-MAT graph (Chakrabarti, Zhan and Faloutsos, SDM 2004), symmetrised, no self loops, no duplicates.

    Edge e (of edge_factor * 2**scale) picks one quadrant per level l with the
    32-bit draw ``splitmix64(seed, e * scale + l) >> 32`` compared against the
    integer thresholds floor(a * 2**32), floor((a+b) * 2**32), floor((a+b+c) * 2**32).
    """
    n = 1 << scale
    m = edge_factor * n
    t1 = np.uint64(int(a * 2**32))
    t2 = np.uint64(int((a + b) * 2**32))
    t3 = np.uint64(int((a + b + c) * 2**32))
    src = np.zeros(m, dtype=np.uint64)
    dst = np.zeros(m, dtype=np.uint64)
    e = np.arange(m, dtype=np.uint64)
    for lvl in range(scale):
        r = splitmix64(seed, e * np.uint64(scale) + np.uint64(lvl)) >> np.uint64(32)
        bit = np.uint64(1) << np.uint64(scale - 1 - lvl)
        down = r >= t2              # quadrants c, d: source bit set
        right = ((r >= t1) & (r < t2)) | (r >= t3)   # quadrants b, d: destination bit set
        src |= np.where(down, bit, np.uint64(0))
        dst |= np.where(right, bit, np.uint64(0))
    keep = src != dst
    src, dst = src[keep], dst[keep]
    return _csr_from_pairs(n, np.concatenate([src, dst]), np.concatenate([dst, src]))


def _as_i64(x: int) -> int:
    """The signed 64-bit integer with the same bits as the unsigned x."""
    x &= 0xFFFFFFFFFFFFFFFF
    return x - (1 << 64) if x >> 63 else x


def splitmix64_torch(seed: int, ctr):
    """SplitMix64 on a torch int64 tensor of counters (any device): the same
    bits as ``splitmix64`` (two's-complement wrap-around for the 64-bit
    products, logical right shifts by masking)."""
    import torch
    z = ctr + 1
    z = z * _as_i64(int(GOLDEN)) + _as_i64(seed)
    z = (z ^ ((z >> 30) & ((1 << 34) - 1))) * _as_i64(int(_M1))
    z = (z ^ ((z >> 27) & ((1 << 37) - 1))) * _as_i64(int(_M2))
    return z ^ ((z >> 31) & ((1 << 33) - 1))


def rmat_csr_torch(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
                   seed: int = 0, device="cpu", chunk: int = 1 << 24):
    """The graph of ``rmat_csr`` generated with torch tensor operations on
    `device` (a GPU makes the large serving pools quick to build).  Returns
    (offsets int64 [n+1], adj int32 [m]) as torch tensors on `device`; the
    values equal rmat_csr's (uint64 offsets, uint32 ids)."""
    import torch
    n = 1 << scale
    m = edge_factor * n
    t1, t2, t3 = int(a * 2**32), int((a + b) * 2**32), int((a + b + c) * 2**32)
    srcs, dsts = [], []
    for lo in range(0, m, chunk):
        e = torch.arange(lo, min(m, lo + chunk), dtype=torch.int64, device=device)
        src = torch.zeros_like(e)
        dst = torch.zeros_like(e)
        for lvl in range(scale):
            r = (splitmix64_torch(seed, e * scale + lvl) >> 32) & 0xFFFFFFFF
            bit = 1 << (scale - 1 - lvl)
            src |= torch.where(r >= t2, bit, 0)
            dst |= torch.where(((r >= t1) & (r < t2)) | (r >= t3), bit, 0)
        keep = src != dst
        srcs.append(src[keep])
        dsts.append(dst[keep])
    src = torch.cat(srcs)
    dst = torch.cat(dsts)
    key = torch.unique(torch.cat([(src << 32) | dst, (dst << 32) | src]))   # sorted, duplicate-free
    s = key >> 32
    adj = (key & 0xFFFFFFFF).to(torch.int32)
    counts = torch.bincount(s, minlength=n)
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=device)
    offsets[1:] = torch.cumsum(counts, 0)
    return offsets, adj


def bfs_sources(offsets: np.ndarray, seed: int, count: int = 3) -> np.ndarray:
    """Source vertex 0 plus ``count`` seeded non-isolated vertices."""
    n = len(offsets) - 1
    deg = np.diff(offsets.astype(np.int64))
    out = [0]
    k = 0
    while len(out) < count + 1 and k < 64 * (count + 1):
        v = int(splitmix64(seed, k) % np.uint64(n))
        k += 1
        if deg[v] > 0 and v not in out:
            out.append(v)
    return np.array(out, dtype=np.uint32)


# ---------------------------------------------------------------------------
# Serving workload: a pool of R-MAT graphs and a stream of BFS requests
# ---------------------------------------------------------------------------

def _unit(seed: int, ctr) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (splitmix64(seed, ctr) >> np.uint64(11)).astype(np.float64) * 2.0**-53


def rmat_pool_scales(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Scales of a graph pool, uniform integers in [lo, hi] (a log-uniform vertex count)."""
    return lo + np.minimum((_unit(seed, np.arange(count)) * (hi - lo + 1)).astype(np.int64), hi - lo)


def serving_requests(offsets_list, count: int, rate: float, seed: int):
    """`count` BFS requests over the graphs whose CSR offsets are listed.

    Graph id uniform over the pool; source the first of up to 64 uniform draws
    with degree > 0 (vertex 0 if none); Poisson arrivals at `rate` per second,
    the first at 0, then exponential gaps -ln(1 - u) / rate.
    Returns (graph ids uint32, sources uint32, arrival offsets float64 seconds)."""
    ng = len(offsets_list)
    gid = np.minimum((_unit(seed, np.arange(count)) * ng).astype(np.int64), ng - 1)
    src = np.zeros(count, dtype=np.uint32)
    for i in range(count):
        off = offsets_list[gid[i]]
        n = len(off) - 1
        draws = splitmix64(seed + 1, np.arange(64, dtype=np.uint64) + np.uint64(64 * i)) % np.uint64(n)
        deg = off[draws.astype(np.int64) + 1] - off[draws.astype(np.int64)]
        hit = np.flatnonzero(deg > 0)
        src[i] = int(draws[hit[0]]) if hit.size else 0
    gaps = -np.log1p(-_unit(seed + 2, np.arange(count))) / float(rate)
    arrival = np.concatenate([[0.0], np.cumsum(gaps[1:])])
    return gid.astype(np.uint32), src, arrival


# ---------------------------------------------------------------------------
# Ray-tracing scene: spheres in the unit box
# ---------------------------------------------------------------------------

def camera_scale(width: int, height: int, vfov_deg: float = 40.0) -> tuple[float, float]:
    """Image-plane half extents of a pinhole camera at distance 1: (tan(vfov/2) * W/H, tan(vfov/2)),
    rounded to float32 once so that every consumer uses the same two numbers."""
    t = np.tan(np.radians(vfov_deg) / 2.0)
    return float(np.float32(t * width / height)), float(np.float32(t))


def sphere_scene(count: int, seed: int = 0, mu: float = -4.0, sigma: float = 0.5) -> dict:
    """``count`` spheres, centres uniform in [0,1]^3, radii exp(N(mu, sigma)), albedo uniform in [0.2, 0.8]^3.

    Returns float32 arrays: centre (count, 3), radius (count,), albedo (count, 3).
    The normal deviate uses the Box-Muller transform on two 24-bit uniforms.
    """
    k = np.arange(count, dtype=np.uint64)
    u = lambda j: ((splitmix64(seed, k * np.uint64(9) + np.uint64(j)) >> np.uint64(40)).astype(np.float64)
                   * 2.0**-24)
    centre = np.stack([u(0), u(1), u(2)], axis=1)
    u1 = np.maximum(u(3), 2.0**-25)
    u2 = u(4)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    radius = np.exp(mu + sigma * z)
    albedo = 0.2 + 0.6 * np.stack([u(5), u(6), u(7)], axis=1)
    return {
        "centre": centre.astype(np.float32),
        "radius": radius.astype(np.float32),
        "albedo": albedo.astype(np.float32),
    }
