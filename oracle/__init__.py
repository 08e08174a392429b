"""CPU oracle for the concurrent FIFO queues (G-LFQ, G-WFQ, G-WFQ-YMC).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never calls it.

What it computes (see ``oracle.h`` for the C entry points):
  * ``seqfifo_run``    the sequential FIFO specification (Section IV's queue model)
  * ``linearizable``   Wing & Gong linearizability search for tiny histories
  * ``check_log``      exactly-once / per-producer-order / no-overtaking checks
  * ``check_tickets``  ticket matching, distinctness and real-time order checks
  * ``mutex_run``      mutex-guarded std::deque on N host threads (timed baseline)
  * ``bfs``            textbook sequential BFS
  * ``render_pixels``  sequential CPU ray tracer (per-pixel radiance)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

OK, FULL, EMPTY = 0, 1, 2
ENQ, DEQ, NOP = 1, 0, 255


class Report(ctypes.Structure):
    _fields_ = [("enq_ok", ctypes.c_int64), ("enq_full", ctypes.c_int64),
                ("deq_ok", ctypes.c_int64), ("deq_empty", ctypes.c_int64),
                ("drained", ctypes.c_int64), ("violations", ctypes.c_int64),
                ("first_kind", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("first_index", ctypes.c_int64)]


class RtScene(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("max_bounces", ctypes.c_int32),
                ("nspheres", ctypes.c_int32), ("cam_x", ctypes.c_float), ("cam_y", ctypes.c_float),
                ("cam_z", ctypes.c_float), ("scale_x", ctypes.c_float), ("scale_y", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("centre", ctypes.c_void_p), ("radius", ctypes.c_void_p),
                ("albedo", ctypes.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, u64, i32, u32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32
        L.orc_seqfifo_run.argtypes = [u64, P, P, i64, P, P, P, P]
        L.orc_seqfifo_run.restype = None
        L.orc_linearizable.argtypes = [i64, P, P, P, P, P, u64, i64]
        L.orc_linearizable.restype = ctypes.c_int
        L.orc_check_log.argtypes = [i64, i64, P, P, P, P, i64, i32, u64, u64, ctypes.POINTER(Report)]
        L.orc_check_log.restype = i64
        L.orc_check_tickets.argtypes = [i64, P, P, P, P, P, P, i32, ctypes.POINTER(Report)]
        L.orc_check_tickets.restype = i64
        L.orc_mutex_run.argtypes = [i32, i64, i64, P, i64, P, u64, i32, P]
        L.orc_mutex_run.restype = ctypes.c_double
        L.orc_bfs.argtypes = [i64, P, P, u32, P]
        L.orc_bfs.restype = i64
        L.orc_render_pixels.argtypes = [ctypes.POINTER(RtScene), P, i64, P, P, i32]
        L.orc_render_pixels.restype = None
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def seqfifo_run(cap, kinds, vals):
    """Replays ops on the sequential FIFO; returns (status int8[n], out uint64[n], final contents)."""
    kinds = np.ascontiguousarray(kinds, dtype=np.uint8)
    vals = np.ascontiguousarray(vals, dtype=np.uint64)
    n = len(kinds)
    status = np.zeros(n, dtype=np.int8)
    out = np.zeros(n, dtype=np.uint64)
    final = np.zeros(n + 1, dtype=np.uint64)
    size = ctypes.c_int64(0)
    lib().orc_seqfifo_run(cap, _p(kinds), _p(vals), n, _p(status), _p(out), _p(final), ctypes.byref(size))
    return status, out, final[: size.value].copy()


def linearizable(op, val, status, call, end, cap=0, max_states=1 << 22):
    """1 linearizable, 0 not, -1 budget exceeded, -2 bad input."""
    op = np.ascontiguousarray(op, dtype=np.uint8)
    val = np.ascontiguousarray(val, dtype=np.uint64)
    status = np.ascontiguousarray(status, dtype=np.int8)
    call = np.ascontiguousarray(call, dtype=np.uint64)
    end = np.ascontiguousarray(end, dtype=np.uint64)
    return lib().orc_linearizable(len(op), _p(op), _p(val), _p(status), _p(call), _p(end), cap, max_states)


def check_log(kind, status, val, drained, prod_shift=32, seq_mask=0xFFFFFFFF, seq_bias=1):
    """Invariant checks on an op-major (K, T) run log.  Returns a dict report."""
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    status = np.ascontiguousarray(status, dtype=np.int8)
    val = np.ascontiguousarray(val, dtype=np.uint64)
    K, T = kind.shape
    drained = np.ascontiguousarray(drained if drained is not None else np.zeros(0), dtype=np.uint64)
    rep = Report()
    lib().orc_check_log(T, K, _p(kind), _p(status), _p(val), _p(drained), len(drained),
                        prod_shift, seq_mask, seq_bias, ctypes.byref(rep))
    return {f: getattr(rep, f) for f, _ in Report._fields_ if f != "pad"}


def check_tickets(kind, status, val, ticket, call=None, end=None, bits=64):
    """Ticket checks (matching, distinct, real-time order) on a run log of any
    shape; the arrays are flattened alike.  Returns a dict report."""
    kind = np.ascontiguousarray(kind, dtype=np.uint8).ravel()
    status = np.ascontiguousarray(status, dtype=np.int8).ravel()
    val = np.ascontiguousarray(val, dtype=np.uint64).ravel()
    ticket = np.ascontiguousarray(ticket, dtype=np.uint64).ravel()
    if call is not None:
        call = np.ascontiguousarray(call, dtype=np.uint64).ravel()
        end = np.ascontiguousarray(end, dtype=np.uint64).ravel()
    rep = Report()
    r = lib().orc_check_tickets(len(kind), _p(kind), _p(status), _p(val), _p(ticket), _p(call), _p(end), bits,
                                ctypes.byref(rep))
    if r < 0:
        raise ValueError("orc_check_tickets: bad arguments")
    return {f: getattr(rep, f) for f, _ in Report._fields_ if f != "pad"}


def mutex_run(mode, T, K, sched=None, producers=0, ops_of=None, cap=0, nthreads=None):
    """Runs the mutex-guarded deque; returns (seconds, counts[4], threads used)."""
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    counts = np.zeros(4, dtype=np.int64)
    sched = None if sched is None else np.ascontiguousarray(sched, dtype=np.uint64)
    ops_of = None if ops_of is None else np.ascontiguousarray(ops_of, dtype=np.int64)
    secs = lib().orc_mutex_run(mode, T, K, _p(sched), producers, _p(ops_of), cap, nthreads, _p(counts))
    return secs, counts, nthreads


def render_pixels(scene: dict, width, height, pixels, max_bounces=8, seed=0, threads=None):
    """Radiance (m, 3) float32 and segment counts of the listed pixel indices."""
    if threads is None:
        threads = os.cpu_count() or 1
    centre = np.ascontiguousarray(scene["centre"], dtype=np.float32)
    radius = np.ascontiguousarray(scene["radius"], dtype=np.float32)
    albedo = np.ascontiguousarray(scene["albedo"], dtype=np.float32)
    cam = scene.get("camera", (0.5, 0.5, -1.5))
    sx, sy = scene["scale"]
    S = RtScene(width, height, max_bounces, len(radius), cam[0], cam[1], cam[2], sx, sy, seed,
                _p(centre), _p(radius), _p(albedo))
    pixels = np.ascontiguousarray(pixels, dtype=np.int64)
    rgb = np.zeros((len(pixels), 3), dtype=np.float32)
    segs = np.zeros(len(pixels), dtype=np.int32)
    lib().orc_render_pixels(ctypes.byref(S), _p(pixels), len(pixels), _p(rgb), _p(segs), threads)
    return rgb, segs


def bfs(offsets, adj, src):
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    adj = np.ascontiguousarray(adj, dtype=np.uint32)
    n = len(offsets) - 1
    dist = np.zeros(n, dtype=np.uint32)
    lib().orc_bfs(n, _p(offsets), _p(adj), int(src), _p(dist))
    return dist
