"""Python binding of libgq: linearizable concurrent FIFO queues on one GB300.

Thin argument marshalling over the C ABI in ``include/gq.h`` and
``include/gq_drivers.h``, ``include/gq_apps.h`` and ``include/gq_serve.h``
(same function names).  Every queue operation runs in
the CUDA kernels of ``libgq.so``; PyTorch only supplies device memory and the
current stream.  There is no CPU fallback: if the library cannot be loaded,
every call raises.

Queue kinds (Section III of "Scalable Concurrent Queues for GPU"):
    GQ_LFQ  G-LFQ, bounded lock-free ring with warp-batched tickets
    GQ_WFQ  G-WFQ, bounded wait-free ring with a cooperative slow path
    GQ_YMC  G-WFQ-YMC, Yang & Mellor-Crummey queue over a pre-allocated pool
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

GQ_LFQ, GQ_WFQ, GQ_YMC = 0, 1, 2
KINDS = {"lfq": GQ_LFQ, "wfq": GQ_WFQ, "ymc": GQ_YMC}
# queue kinds whose device code is complete
READY_KINDS = ["lfq", "wfq", "ymc"]
GQ_OK, GQ_FULL, GQ_EMPTY = 0, 1, 2
GQ_ERR_INVALID, GQ_ERR_NOMEM, GQ_ERR_CUDA, GQ_ERR_TIMEOUT = -1, -2, -3, -4
GQ_ERR_POOL_EXHAUSTED, GQ_ERR_TOO_MANY_THREADS, GQ_ERR_RESERVED_VALUE = -5, -6, -7
GQ_RUN_PAIRS, GQ_RUN_MIXED, GQ_RUN_SPLIT = 0, 1, 2
GQ_DUE_WAIT_OFF = 0xFFFFFFFF
GQ_PEAK_SAME_ADDR_FAA, GQ_PEAK_COALESCED_CAS, GQ_PEAK_SCATTERED_CAS, GQ_PEAK_COALESCED_LOAD = 0, 1, 2, 3
GQ_PEAK_SPREAD_FAA, GQ_PEAK_PACKED_FAA = 4, 5
(GQ_CNT_ENQ_OK, GQ_CNT_ENQ_FULL, GQ_CNT_DEQ_OK, GQ_CNT_DEQ_EMPTY, GQ_CNT_SUM_ENQ, GQ_CNT_SUM_DEQ,
 GQ_CNT_ERRORS) = range(7)
# event counters of the counting kernels (gq_run / gq_run_multi with opcount=)
OC_NAMES = ["tickets", "faa", "cas", "cas_fail", "rmw", "threshold", "catchup", "burned", "loads", "slow",
            "spin", "marked"]
GQ_OC_N = len(OC_NAMES)

# Every symbol the headers in include/ declare.
EXPORTS = [
    "gq_workspace_bytes", "gq_create", "gq_destroy", "gq_reset", "gq_enqueue_batch", "gq_dequeue_batch",
    "gq_sync_status", "gq_device_view", "gq_info", "gq_status_str", "gq_get_stats",
    "gq_run", "gq_run_sequence", "gq_drain", "gq_atomic_peak", "gq_fifo_static_roundtrip",
    "gq_bfs", "gq_render_workspace_bytes", "gq_render", "gq_multi_prepare", "gq_run_multi",
    "gq_bfs_batch_workspace_bytes", "gq_bfs_batch", "gq_serve", "gq_wavefaa_probe",
]
GQ_VIEW_BYTES = 512


class GqError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__("%s: %s (%d)" % (what, status_str(status), status))


class gq_options(ctypes.Structure):
    _fields_ = [("cycle_bits", ctypes.c_uint32), ("patience_enq", ctypes.c_uint32),
                ("patience_deq", ctypes.c_uint32), ("patience_set", ctypes.c_uint32),
                ("help_delay", ctypes.c_uint32), ("batch_width", ctypes.c_uint32),
                ("backoff_ns", ctypes.c_uint32), ("due_wait", ctypes.c_uint32),
                ("patience_stretch", ctypes.c_uint32), ("reserved_opt", ctypes.c_uint32),
                ("start_ticket", ctypes.c_uint64)]


class gq_run_args(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("threads", ctypes.c_uint32), ("block", ctypes.c_uint32),
                ("ops", ctypes.c_uint32), ("producers", ctypes.c_uint32), ("delay_ns", ctypes.c_uint32),
                ("total_ops", ctypes.c_uint64), ("d_sched", ctypes.c_void_p), ("d_status", ctypes.c_void_p),
                ("d_val", ctypes.c_void_p), ("d_call", ctypes.c_void_p), ("d_end", ctypes.c_void_p),
                ("d_counts", ctypes.c_void_p), ("d_ticket", ctypes.c_void_p), ("d_opcount", ctypes.c_void_p)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Loads libgq.so (building it first if it is missing or stale).  Raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = ctypes.CDLL(path)
    P, i32, u32, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
    sig = {
        "gq_workspace_bytes": [i32, u64, u32, u32, P, P],
        "gq_create": [i32, u64, u32, u32, P, P, P, P],
        "gq_destroy": [P],
        "gq_reset": [P, P],
        "gq_enqueue_batch": [P, P, u64, P, P, P],
        "gq_dequeue_batch": [P, P, u64, P, P, P],
        "gq_sync_status": [P, P],
        "gq_device_view": [P, P],
        "gq_info": [P, P, P],
        "gq_status_str": [i32],
        "gq_get_stats": [P, P],
        "gq_run": [P, P, P],
        "gq_run_sequence": [P, P, P, u64, P, P, P],
        "gq_drain": [P, P, u64, P, P],
        "gq_atomic_peak": [i32, u32, u32, u32, P, u64, P, P],
        "gq_fifo_static_roundtrip": [P, u64, P, P, P],
        "gq_bfs": [P, P, u64, P, P, u32, P, P, P],
        "gq_render_workspace_bytes": [P, P],
        "gq_render": [P, P, P, P, P, P],
        "gq_multi_prepare": [P, u32, P, P, P],
        "gq_run_multi": [P, P, P],
        "gq_bfs_batch_workspace_bytes": [u32, P],
        "gq_bfs_batch": [P, P, u32, u32, P, P, u32, P, P, P],
        "gq_serve": [P, P],
        "gq_wavefaa_probe": [P, u32, u32, P, P, P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name == "gq_status_str" else ctypes.c_int
    _lib = L
    return L


def status_str(s: int) -> str:
    return load().gq_status_str(int(s)).decode()


def _check(s: int, what: str) -> int:
    if s < 0:
        raise GqError(s, what)
    return s


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _need(t, n: int, elem: int, what: str) -> None:
    """Checks a buffer before its address crosses the C ABI: a contiguous CUDA
    tensor with room for n elements of `elem` bytes.  Raw integer addresses
    and None (nullable arguments) pass unchecked."""
    if t is None or isinstance(t, int):
        return
    if not getattr(t, "is_cuda", False):
        raise GqError(GQ_ERR_INVALID, what + " (not a CUDA tensor)")
    if not t.is_contiguous():
        raise GqError(GQ_ERR_INVALID, what + " (not contiguous)")
    if t.numel() * t.element_size() < n * elem:
        raise GqError(GQ_ERR_INVALID, what + " (holds %d bytes, needs %d)" % (t.numel() * t.element_size(), n * elem))


_ELEM_BYTES: dict = {}   # payload width of the handles made through this module


def _elem_bytes(h: int) -> int:
    """Payload width of a queue handle (remembered from gq_create, else read
    from its device view)."""
    eb = _ELEM_BYTES.get(h)
    if eb is None:
        buf = (ctypes.c_uint8 * GQ_VIEW_BYTES)()
        _check(load().gq_device_view(h, buf), "gq_device_view")
        eb = int.from_bytes(bytes(buf[4:8]), "little")
    return eb


def _stream(stream=None) -> int | None:
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


# ---------------------------------------------------------------------------
# C-ABI entry points (same names, raise GqError on a negative status)
# ---------------------------------------------------------------------------

def gq_workspace_bytes(kind: int, capacity: int, elem_bytes: int, max_threads: int, opt: gq_options | None = None) -> int:
    out = ctypes.c_uint64(0)
    _check(load().gq_workspace_bytes(kind, capacity, elem_bytes, max_threads,
                                     ctypes.byref(opt) if opt else None, ctypes.byref(out)), "gq_workspace_bytes")
    return out.value


def gq_create(kind: int, capacity: int, elem_bytes: int, max_threads: int, opt: gq_options | None = None,
              workspace=None, stream=None) -> int:
    h = ctypes.c_void_p(0)
    _check(load().gq_create(kind, capacity, elem_bytes, max_threads, ctypes.byref(opt) if opt else None,
                            _ptr(workspace), _stream(stream), ctypes.byref(h)), "gq_create")
    _ELEM_BYTES[h.value] = elem_bytes
    return h.value


def gq_destroy(h: int) -> None:
    _ELEM_BYTES.pop(h, None)
    _check(load().gq_destroy(h), "gq_destroy")


def gq_reset(h: int, stream=None) -> None:
    _check(load().gq_reset(h, _stream(stream)), "gq_reset")


def gq_enqueue_batch(h: int, items, n: int | None = None, status=None, num_ok=None, stream=None) -> None:
    eb = _elem_bytes(h)
    n = items.numel() * items.element_size() // eb if n is None else n
    _need(items, n, eb, "gq_enqueue_batch: items")
    _need(status, n, 1, "gq_enqueue_batch: status")
    _need(num_ok, 1, 8, "gq_enqueue_batch: num_ok")
    _check(load().gq_enqueue_batch(h, _ptr(items), n, _ptr(status), _ptr(num_ok), _stream(stream)),
           "gq_enqueue_batch")


def gq_dequeue_batch(h: int, out, n: int | None = None, status=None, num_ok=None, stream=None) -> None:
    eb = _elem_bytes(h)
    n = out.numel() * out.element_size() // eb if n is None else n
    _need(out, n, eb, "gq_dequeue_batch: out")
    _need(status, n, 1, "gq_dequeue_batch: status")
    _need(num_ok, 1, 8, "gq_dequeue_batch: num_ok")
    _check(load().gq_dequeue_batch(h, _ptr(out), n, _ptr(status), _ptr(num_ok), _stream(stream)),
           "gq_dequeue_batch")


def gq_sync_status(h: int, stream=None) -> int:
    """Synchronises the stream and returns (and clears) the latched device error status."""
    return load().gq_sync_status(h, _stream(stream))


class gq_stats(ctypes.Structure):
    _fields_ = [("slow_requests", ctypes.c_uint64), ("helps", ctypes.c_uint64),
                ("global_cas_failures", ctypes.c_uint64), ("slow_rounds_tail", ctypes.c_uint64),
                ("slow_rounds_head", ctypes.c_uint64), ("max_help_iterations", ctypes.c_uint64),
                ("aq_head", ctypes.c_uint64), ("aq_tail", ctypes.c_uint64), ("fq_head", ctypes.c_uint64),
                ("fq_tail", ctypes.c_uint64), ("aq_slow_pending", ctypes.c_uint64),
                ("fq_slow_pending", ctypes.c_uint64)]


def gq_get_stats(h: int) -> dict:
    s = gq_stats()
    _check(load().gq_get_stats(h, ctypes.byref(s)), "gq_get_stats")
    return {f: getattr(s, f) for f, _ in gq_stats._fields_}


def gq_info(h: int) -> tuple[int, bool]:
    b, o = ctypes.c_uint64(0), ctypes.c_int(0)
    _check(load().gq_info(h, ctypes.byref(b), ctypes.byref(o)), "gq_info")
    return b.value, bool(o.value)


def gq_run(h: int, mode: int, threads: int, block: int = 256, ops: int = 0, producers: int = 0,
           total_ops: int = 0, sched=None, status=None, val=None, call=None, end=None, counts=None,
           delay_ns: int = 0, stream=None, ticket=None, opcount=None) -> None:
    _need(opcount, GQ_OC_N, 8, "gq_run: opcount")
    _need(counts, 8, 8, "gq_run: counts")
    a = gq_run_args(mode, threads, block, ops, producers, delay_ns, total_ops, _ptr(sched), _ptr(status),
                    _ptr(val), _ptr(call), _ptr(end), _ptr(counts), _ptr(ticket), _ptr(opcount))
    _check(load().gq_run(h, ctypes.byref(a), _stream(stream)), "gq_run")


def gq_run_sequence(h: int, kind, val, status, out, stream=None) -> None:
    _check(load().gq_run_sequence(h, _ptr(kind), _ptr(val), kind.numel(), _ptr(status), _ptr(out),
                                  _stream(stream)), "gq_run_sequence")


def gq_drain(h: int, out, count, max_items: int | None = None, stream=None) -> None:
    m = out.numel() if max_items is None else max_items
    _check(load().gq_drain(h, _ptr(out), m, _ptr(count), _stream(stream)), "gq_drain")


def gq_atomic_peak(pattern: int, blocks: int, threads: int, iters: int, buf, sink, stream=None) -> None:
    _check(load().gq_atomic_peak(pattern, blocks, threads, iters, _ptr(buf), buf.numel(), _ptr(sink),
                                 _stream(stream)), "gq_atomic_peak")


def gq_wavefaa_probe(take, width: int, counters, tickets, stream=None) -> None:
    """Test hook for WaveFAA: thread t takes a ticket on counter take[t]-1 (1 or 2), batch width `width`."""
    _check(load().gq_wavefaa_probe(_ptr(take), take.numel(), width, _ptr(counters), _ptr(tickets), _stream(stream)),
           "gq_wavefaa_probe")


def gq_fifo_static_roundtrip(items, out, num_out, n: int | None = None, stream=None) -> None:
    """FIFO round trip on the library's static device array (no allocation; n <= 65536)."""
    n = items.numel() if n is None else n
    _need(items, n, 8, "gq_fifo_static_roundtrip: items")
    _need(out, n, 8, "gq_fifo_static_roundtrip: out")
    _need(num_out, 1, 8, "gq_fifo_static_roundtrip: num_out")
    _check(load().gq_fifo_static_roundtrip(_ptr(items), n, _ptr(out), _ptr(num_out), _stream(stream)),
           "gq_fifo_static_roundtrip")


GQ_BFS_UNREACHED = 0xFFFFFFFF


def gq_bfs(q_a: int, q_b: int, offsets, adj, src: int, dist, stats=None, stream=None) -> None:
    """Level-synchronous BFS with two alternating frontier queues (4-byte queues of one kind)."""
    _check(load().gq_bfs(q_a, q_b, offsets.numel() - 1, _ptr(offsets), _ptr(adj), src, _ptr(dist), _ptr(stats),
                         _stream(stream)), "gq_bfs")


class gq_bfs_instance(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("d_offsets", ctypes.c_void_p), ("d_adj", ctypes.c_void_p),
                ("d_dist", ctypes.c_void_p), ("src", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class BatchBfs:
    """Many BFS instances in one persistent launch (one per thread-block cluster at a time)."""

    def __init__(self, kind, graphs, sources, slots=64, cluster_blocks=4, max_levels=64):
        import numpy as np
        import torch
        self.torch = torch
        self.kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        self.graphs = []
        inst = (gq_bfs_instance * len(graphs))()
        nmax = 1
        for i, ((off, adj), src) in enumerate(zip(graphs, sources)):
            d_off = torch.from_numpy(off.view(np.int64)).cuda()
            d_adj = torch.from_numpy(adj.view(np.int32)).cuda()
            dist = torch.empty(len(off) - 1, dtype=torch.int32, device="cuda")
            self.graphs.append((d_off, d_adj, dist))
            inst[i] = gq_bfs_instance(len(off) - 1, d_off.data_ptr(), d_adj.data_ptr(), dist.data_ptr(), int(src), 0)
            nmax = max(nmax, len(off) - 1)
        self.ninst = len(graphs)
        self.d_inst = torch.frombuffer(bytearray(bytes(inst)), dtype=torch.uint8).cuda()
        sizes = np.array([len(g[0]) - 1 for g in graphs])
        self.d_order = torch.from_numpy(np.argsort(-sizes, kind="stable").astype(np.int32)).cuda()
        self.slots, self.cluster_blocks = slots, cluster_blocks
        if self.kind == GQ_YMC:
            cap = 3 * nmax + 64 * (max_levels + 1) + (1 << 17)
        else:
            cap = min(1 << max(12, (nmax - 1).bit_length()), 1 << 23)
        self.idq = Queue(GQ_LFQ, 1 << max(1, (self.ninst - 1).bit_length()), 4, max(slots, 32))
        self.frontier = [Queue(self.kind, cap, 4, cluster_blocks * 256) for _ in range(2 * slots)]
        ws = ctypes.c_uint64(0)
        _check(load().gq_bfs_batch_workspace_bytes(slots, ctypes.byref(ws)), "gq_bfs_batch_workspace_bytes")
        self.ws = torch.empty(ws.value, dtype=torch.uint8, device="cuda")
        self.stats = torch.zeros(4, dtype=torch.int64, device="cuda")

    def run(self, stream=None):
        arr = (ctypes.c_void_p * len(self.frontier))(*[q.handle for q in self.frontier])
        _check(load().gq_bfs_batch(self.idq.handle, arr, self.slots, self.cluster_blocks, _ptr(self.d_inst),
                                   _ptr(self.d_order), self.ninst, _ptr(self.ws), _ptr(self.stats),
                                   _stream(stream)), "gq_bfs_batch")

    def dists(self):
        return [g[2] for g in self.graphs]


class gq_multi_args(ctypes.Structure):
    _fields_ = [("nqueues", ctypes.c_uint32), ("threads_per_queue", ctypes.c_uint32),
                ("producers_per_queue", ctypes.c_uint32), ("block", ctypes.c_uint32), ("blocks", ctypes.c_uint32),
                ("kind", ctypes.c_uint32), ("elem_bytes", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("ops_per_queue", ctypes.c_uint64), ("d_counts", ctypes.c_void_p), ("d_status", ctypes.c_void_p),
                ("d_val", ctypes.c_void_p), ("d_ticket", ctypes.c_void_p), ("d_opcount", ctypes.c_void_p)]


def gq_multi_prepare(handles, views, tune: gq_options | None = None, stream=None) -> None:
    arr = (ctypes.c_void_p * len(handles))(*handles)
    _check(load().gq_multi_prepare(arr, len(handles), _ptr(views), ctypes.byref(tune) if tune else None,
                                   _stream(stream)), "gq_multi_prepare")


def gq_run_multi(views, nqueues: int, kind: int, elem_bytes: int, threads_per_queue: int, producers_per_queue: int,
                 ops_per_queue: int, counts, block: int = 256, blocks: int = 0, stream=None, status=None, val=None,
                 ticket=None, opcount=None) -> None:
    """Producer/consumer workload on every queue of `views` in one persistent launch.  status / val /
    ticket (recorder) hold nqueues * K * threads_per_queue entries, K = ceil(ops_per_queue /
    threads_per_queue); opcount (GQ_OC_N words) selects the counting kernel."""
    K = -(-ops_per_queue // threads_per_queue)
    n = nqueues * K * threads_per_queue
    _need(counts, 8, 8, "gq_run_multi: counts")
    _need(status, n, 1, "gq_run_multi: status")
    _need(val, n, 8, "gq_run_multi: val")
    _need(ticket, n, 8, "gq_run_multi: ticket")
    _need(opcount, GQ_OC_N, 8, "gq_run_multi: opcount")
    a = gq_multi_args(nqueues, threads_per_queue, producers_per_queue, block, blocks, kind, elem_bytes, 0,
                      ops_per_queue, _ptr(counts), _ptr(status), _ptr(val), _ptr(ticket), _ptr(opcount))
    _check(load().gq_run_multi(_ptr(views), ctypes.byref(a), _stream(stream)), "gq_run_multi")


class MultiQueue:
    """Q independent queues of one kind, for the batched persistent driver."""

    def __init__(self, kind, capacities, elem_bytes: int = 8, max_threads: int = 1024, **options):
        import torch
        self.kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        self.elem_bytes = elem_bytes
        self.queues = [Queue(self.kind, int(c), elem_bytes, max_threads, **options) for c in capacities]
        self.handles = [q.handle for q in self.queues]
        self.views = torch.empty(len(self.queues) * GQ_VIEW_BYTES, dtype=torch.uint8, device="cuda")
        self.prepare()

    def prepare(self, batch_width: int = 0, backoff_ns: int | None = None, patience=None, help_delay: int = 0,
                due_wait: int = 0, patience_stretch: int = 0, stream=None):
        tune = None
        if (batch_width or backoff_ns is not None or patience is not None or help_delay or due_wait
                or patience_stretch):
            tune = gq_options(batch_width=batch_width, backoff_ns=backoff_ns or 0, help_delay=help_delay,
                              due_wait=due_wait, patience_stretch=patience_stretch)
            if patience is not None:
                tune.patience_enq, tune.patience_deq, tune.patience_set = patience[0], patience[1], 1
        gq_multi_prepare(self.handles, self.views, tune, stream)

    def reset(self, stream=None):
        for q in self.queues:
            q.reset(stream)

    def run(self, threads_per_queue, producers_per_queue, ops_per_queue, counts, block=256, blocks=0, stream=None,
            **record):
        """record: status= / val= / ticket= (recorder) or opcount= (counting kernel), see gq_run_multi."""
        gq_run_multi(self.views, len(self.queues), self.kind, self.elem_bytes, threads_per_queue, producers_per_queue,
                     ops_per_queue, counts, block, blocks, stream, **record)

    def run_per_call(self, threads_per_queue, producers_per_queue, ops_per_queue, counts, block=256, stream=None):
        """The plain form: one split-workload launch per queue, one after another."""
        for q in self.queues:
            gq_run(q.handle, GQ_RUN_SPLIT, threads_per_queue, block=block, producers=producers_per_queue,
                   total_ops=ops_per_queue, counts=counts, stream=stream)

    def close(self):
        for q in self.queues:
            q.close()


class gq_rt_scene(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("height", ctypes.c_uint32), ("tiles_x", ctypes.c_uint32),
                ("tiles_y", ctypes.c_uint32), ("max_bounces", ctypes.c_uint32), ("nspheres", ctypes.c_uint32),
                ("cam_x", ctypes.c_float), ("cam_y", ctypes.c_float), ("cam_z", ctypes.c_float),
                ("scale_x", ctypes.c_float), ("scale_y", ctypes.c_float), ("reserved", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("d_centre", ctypes.c_void_p), ("d_radius", ctypes.c_void_p),
                ("d_albedo", ctypes.c_void_p)]


def gq_render_workspace_bytes(scene: gq_rt_scene) -> int:
    out = ctypes.c_uint64(0)
    _check(load().gq_render_workspace_bytes(ctypes.byref(scene), ctypes.byref(out)), "gq_render_workspace_bytes")
    return out.value


def gq_render(tiles, scene: gq_rt_scene, workspace, image, stats=None, stream=None) -> None:
    """Tile-based wavefront ray tracing; tiles: list of queue handles (tiles_x * tiles_y)."""
    arr = (ctypes.c_void_p * len(tiles))(*tiles)
    _check(load().gq_render(arr, ctypes.byref(scene), _ptr(workspace), _ptr(image), _ptr(stats), _stream(stream)),
           "gq_render")


class Renderer:
    """Tile queues, workspace and scene arrays for gq_render (device memory from torch)."""

    def __init__(self, kind, scene: dict, width: int, height: int, tiles=(8, 8), max_bounces=8, seed=0,
                 max_threads=1 << 19):
        import math
        import torch
        self.torch = torch
        self.centre = torch.as_tensor(scene["centre"], dtype=torch.float32).reshape(-1).contiguous().cuda()
        self.radius = torch.as_tensor(scene["radius"], dtype=torch.float32).contiguous().cuda()
        self.albedo = torch.as_tensor(scene["albedo"], dtype=torch.float32).reshape(-1).contiguous().cuda()
        cam = scene.get("camera", (0.5, 0.5, -1.5))
        sx, sy = scene["scale"]
        ns = self.radius.numel()
        self.scene = gq_rt_scene(width, height, tiles[0], tiles[1], max_bounces, ns, cam[0], cam[1], cam[2], sx, sy, 0,
                                 seed, self.centre.data_ptr() if ns else None, self.radius.data_ptr() if ns else None,
                                 self.albedo.data_ptr() if ns else None)
        tw, th = -(-width // tiles[0]), -(-height // tiles[1])
        per_tile = tw * th
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        if k == GQ_YMC:
            cap = (max_bounces + 1) * per_tile + (1 << 14)
        else:
            cap = 1 << max(12, (per_tile - 1).bit_length())
        self.queues = [Queue(k, cap, 4, max_threads) for _ in range(tiles[0] * tiles[1])]
        self.ws = torch.empty(gq_render_workspace_bytes(self.scene), dtype=torch.uint8, device="cuda")
        self.image = torch.zeros((height, width, 3), dtype=torch.float32, device="cuda")
        self.stats = torch.zeros(4, dtype=torch.int64, device="cuda")

    def render(self, stream=None):
        for q in self.queues:
            q.reset(stream)
        gq_render([q.handle for q in self.queues], self.scene, self.ws, self.image, self.stats, stream)
        return self.image


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------

class Queue:
    """Owns one libgq queue handle.  All methods are asynchronous on the current stream."""

    def __init__(self, kind, capacity: int, elem_bytes: int = 8, max_threads: int = 1 << 20,
                 use_torch_memory: bool = False, **options):
        self.kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        self.capacity = capacity
        self.elem_bytes = elem_bytes
        self.max_threads = max_threads
        self.opt = gq_options(**options) if options else None
        if "patience_enq" in options or "patience_deq" in options:
            self.opt.patience_set = 1
        self._ws = None
        if use_torch_memory:
            import torch
            nbytes = gq_workspace_bytes(self.kind, capacity, elem_bytes, max_threads, self.opt)
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            addr = (self._ws.data_ptr() + 255) // 256 * 256
            self.handle = gq_create(self.kind, capacity, elem_bytes, max_threads, self.opt, addr)
        else:
            self.handle = gq_create(self.kind, capacity, elem_bytes, max_threads, self.opt)

    def reset(self, stream=None):
        gq_reset(self.handle, stream)

    def enqueue(self, items, status=None, num_ok=None, stream=None):
        gq_enqueue_batch(self.handle, items, None, status, num_ok, stream)

    def dequeue(self, out, status=None, num_ok=None, stream=None):
        gq_dequeue_batch(self.handle, out, None, status, num_ok, stream)

    def stats(self) -> dict:
        return gq_get_stats(self.handle)

    def sync_status(self, stream=None) -> int:
        return gq_sync_status(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            gq_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- serving (include/gq_serve.h) ----
GQ_SERVE_PERSISTENT, GQ_SERVE_PER_REQUEST, GQ_SERVE_ADAPTIVE = 0, 1, 2
SERVE_MODES = {"persistent": GQ_SERVE_PERSISTENT, "per_request": GQ_SERVE_PER_REQUEST, "adaptive": GQ_SERVE_ADAPTIVE}


class gq_serve_config(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("mode", ctypes.c_uint32), ("slots", ctypes.c_uint32),
                ("cluster_blocks", ctypes.c_uint32), ("budget_bytes", ctypes.c_uint64),
                ("wait_limit_s", ctypes.c_double), ("ngraphs", ctypes.c_uint32), ("nrequests", ctypes.c_uint32),
                ("graphs", ctypes.c_void_p), ("req_graph", ctypes.c_void_p), ("req_src", ctypes.c_void_p),
                ("req_arrival_s", ctypes.c_void_p), ("req_out", ctypes.c_void_p),
                ("switch_backlog", ctypes.c_uint32), ("gang_clusters", ctypes.c_uint32),
                ("gang_min_vertices", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class gq_serve_result(ctypes.Structure):
    _fields_ = [("latency_s", ctypes.c_void_p), ("wall_s", ctypes.c_double), ("peak_state_bytes", ctypes.c_uint64),
                ("admission_waits", ctypes.c_uint64), ("edges_scanned", ctypes.c_uint64),
                ("persistent_requests", ctypes.c_uint64), ("slots_used", ctypes.c_uint32),
                ("status", ctypes.c_int32), ("gang_requests", ctypes.c_uint64)]


def gq_serve(kind, graphs, req_graph, req_src, arrival_s, mode="persistent", slots: int = 0,
             cluster_blocks: int = 4, budget_bytes: int = 32 << 30, outs=None, wait_limit_s: float = 0.0,
             switch_backlog: int = 0, gang_clusters: int = 0, gang_min_vertices: int = 0) -> dict:
    """Serves BFS requests (include/gq_serve.h).

    graphs: list of (d_offsets int64, d_adj int32) device tensors (CSR).
    req_graph, req_src: request graph ids and source vertices; arrival_s:
    non-decreasing arrival offsets in seconds.  outs: optional list of device
    int32 tensors (or None entries) receiving each request's distances.
    Returns latencies (numpy, seconds) and the run's counters."""
    import numpy as np
    lib = load()
    kind = KINDS[kind] if isinstance(kind, str) else int(kind)
    mode = SERVE_MODES[mode] if isinstance(mode, str) else int(mode)
    g = (gq_bfs_instance * len(graphs))()
    for i, (off, adj) in enumerate(graphs):
        g[i] = gq_bfs_instance(off.numel() - 1, off.data_ptr(), adj.data_ptr(), None, 0, 0)
    rg = np.ascontiguousarray(req_graph, dtype=np.uint32)
    rs = np.ascontiguousarray(req_src, dtype=np.uint32)
    ra = np.ascontiguousarray(arrival_s, dtype=np.float64)
    n = len(rg)
    if len(rs) != n or len(ra) != n:
        raise ValueError("request arrays differ in length")
    out_arr = None
    if outs is not None:
        out_arr = (ctypes.c_void_p * n)(*[None if o is None else o.data_ptr() for o in outs])
    lat = np.full(n, -1.0)
    cfg = gq_serve_config(kind, mode, slots, cluster_blocks, budget_bytes, wait_limit_s, len(graphs), n,
                          ctypes.cast(g, ctypes.c_void_p), rg.ctypes.data, rs.ctypes.data, ra.ctypes.data,
                          None if out_arr is None else ctypes.cast(out_arr, ctypes.c_void_p), switch_backlog,
                          gang_clusters, gang_min_vertices, 0)
    res = gq_serve_result(lat.ctypes.data, 0.0, 0, 0, 0, 0, 0, 0, 0)
    _check(lib.gq_serve(ctypes.byref(cfg), ctypes.byref(res)), "gq_serve")
    return {"latency_s": lat, "wall_s": res.wall_s, "peak_state_bytes": res.peak_state_bytes,
            "admission_waits": res.admission_waits, "edges_scanned": res.edges_scanned,
            "persistent_requests": res.persistent_requests, "slots_used": res.slots_used,
            "gang_requests": res.gang_requests}
