"""libgq loads and exports every symbol its headers declare; host-side argument
validation and workspace layout need no GPU (CPU only)."""
import ctypes
import os
import re

import pytest

import paper_2606_01693_gb300 as gq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in ("gq.h", "gq_drivers.h", "gq_apps.h", "gq_serve.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:int|const char\*|void)\s+(gq_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol():
    L = gq.load()
    declared = _declared_symbols()
    assert declared, "no declarations parsed"
    assert declared == set(gq.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


def test_status_strings():
    assert gq.status_str(0) == "ok"
    assert gq.status_str(gq.GQ_ERR_TIMEOUT) == "bounded device loop expired"


@pytest.mark.parametrize("kind,cap,elem,thr", [
    (gq.GQ_LFQ, 3, 8, 1),         # capacity not a power of two
    (gq.GQ_LFQ, 1, 8, 1),         # capacity < 2
    (gq.GQ_LFQ, 1 << 32, 8, 1),   # above the 32-bit index field
    (gq.GQ_WFQ, 1 << 24, 8, 1),   # above the 24-bit index field
    (gq.GQ_LFQ, 16, 2, 1),        # element size
    (gq.GQ_YMC, 1, 8, 1),         # pool too small
    (7, 16, 8, 1),                # kind
    (gq.GQ_LFQ, 16, 8, 0),        # no threads
])
def test_invalid_arguments_rejected(kind, cap, elem, thr):
    with pytest.raises(gq.GqError) as ei:
        gq.gq_workspace_bytes(kind, cap, elem, thr)
    assert ei.value.status == gq.GQ_ERR_INVALID
    h = ctypes.c_void_p(0)
    assert gq.load().gq_create(kind, cap, elem, thr, None, None, None, ctypes.byref(h)) == gq.GQ_ERR_INVALID
    assert not h.value


def test_wfq_cycle_soundness_bound():
    # Lemma "Modular cycle correctness": sound iff R > D k / n + 6.
    # R = 2^4 = 16, D = 64, n = 64: k = 9 gives 9 + 6 = 15 < 16 (ok), k = 10 gives 16 (rejected).
    ok = gq.gq_options(cycle_bits=4, help_delay=64)
    assert gq.gq_workspace_bytes(gq.GQ_WFQ, 64, 8, 9, ok) > 0
    with pytest.raises(gq.GqError) as ei:
        gq.gq_workspace_bytes(gq.GQ_WFQ, 64, 8, 10, ok)
    assert ei.value.status == gq.GQ_ERR_TOO_MANY_THREADS


def test_bad_options_rejected():
    for o in (gq.gq_options(batch_width=3), gq.gq_options(batch_width=64), gq.gq_options(cycle_bits=32),
              gq.gq_options(start_ticket=5), gq.gq_options(patience_stretch=4097),
              gq.gq_options(reserved_opt=1)):
        with pytest.raises(gq.GqError):
            gq.gq_workspace_bytes(gq.GQ_LFQ, 16, 8, 1, o)
    # the patience stretch is a G-WFQ option; its bound holds for every kind
    assert gq.gq_workspace_bytes(gq.GQ_WFQ, 16, 8, 1, gq.gq_options(patience_stretch=4096)) > 0
    with pytest.raises(gq.GqError):
        gq.gq_workspace_bytes(gq.GQ_WFQ, 16, 8, 1, gq.gq_options(patience_stretch=4097))


def test_options_layout_matches_header():
    # gq_options as include/gq.h declares it: nine 32-bit fields, then the 64-bit start ticket
    assert ctypes.sizeof(gq.gq_options) == 48
    assert gq.gq_options.start_ticket.offset == 40
    assert gq.gq_options.patience_stretch.offset == 32


def test_workspace_grows_with_capacity_and_records():
    a = gq.gq_workspace_bytes(gq.GQ_LFQ, 1 << 10, 8, 1)
    b = gq.gq_workspace_bytes(gq.GQ_LFQ, 1 << 20, 8, 1)
    # 2 rings x 2n slots x 8 B + n payloads x 8 B
    assert b - a == (2 * 2 * 8 + 8) * ((1 << 20) - (1 << 10))
    w1 = gq.gq_workspace_bytes(gq.GQ_WFQ, 1 << 10, 8, 1024)
    w2 = gq.gq_workspace_bytes(gq.GQ_WFQ, 1 << 10, 8, 2048)
    assert w2 - w1 == 2 * 1024 * (128 + 8)    # one 128-byte record and one help cursor per thread per ring
    y = gq.gq_workspace_bytes(gq.GQ_YMC, 1000, 8, 256)
    assert y >= 3 * 1001 * 8 + 256 * 128
    for v in (a, b, w1, w2, y):
        assert v % 256 == 0


def _serve_cfg(**kw):
    """A serving configuration with fake device addresses (only validated, never dereferenced)."""
    import numpy as np
    g = (gq.gq_bfs_instance * 2)(gq.gq_bfs_instance(100, 0x10000, 0x20000, None, 0, 0),
                                 gq.gq_bfs_instance(50, 0x30000, 0x40000, None, 0, 0))
    rg = np.array(kw.pop("req_graph", [0, 1, 0]), dtype=np.uint32)
    rs = np.array(kw.pop("req_src", [3, 49, 99]), dtype=np.uint32)
    ra = np.array(kw.pop("arrival", [0.0, 0.1, 0.2]), dtype=np.float64)
    keep = [g, rg, rs, ra]
    cfg = gq.gq_serve_config(kind=kw.pop("kind", 0), mode=kw.pop("mode", 0), slots=0,
                             cluster_blocks=kw.pop("cluster_blocks", 2), budget_bytes=kw.pop("budget", 1 << 30),
                             wait_limit_s=kw.pop("wait", 0.0), ngraphs=kw.pop("ngraphs", 2), nrequests=len(rg),
                             graphs=ctypes.cast(g, ctypes.c_void_p).value, req_graph=rg.ctypes.data,
                             req_src=rs.ctypes.data, req_arrival_s=ra.ctypes.data, req_out=None,
                             gang_clusters=kw.pop("gang", 0), reserved=kw.pop("reserved", 0))
    lat = np.zeros(len(rg))
    res = gq.gq_serve_result(latency_s=lat.ctypes.data)
    keep.append(lat)
    return cfg, res, keep


@pytest.mark.parametrize("change", [
    {"kind": 7}, {"mode": 3}, {"cluster_blocks": 3}, {"cluster_blocks": 32}, {"req_graph": [0, 2, 0]}, {"req_src": [3, 50, 99]},
    {"arrival": [0.0, 0.2, 0.1]}, {"arrival": [0.0, float("nan"), 0.2]}, {"budget": 0}, {"wait": -1.0},
    {"ngraphs": 0}, {"gang": 65}, {"reserved": 1},
])
def test_serve_rejects_bad_config(change):
    cfg, res, keep = _serve_cfg(**change)
    assert gq.load().gq_serve(ctypes.byref(cfg), ctypes.byref(res)) == gq.GQ_ERR_INVALID
    assert gq.load().gq_serve(None, ctypes.byref(res)) == gq.GQ_ERR_INVALID
    assert gq.load().gq_serve(ctypes.byref(cfg), None) == gq.GQ_ERR_INVALID


def test_atomic_peak_arguments_validated():
    L = gq.load()
    sink = ctypes.c_void_p(0x1000)   # never dereferenced: every call below fails validation first
    buf = ctypes.c_void_p(0x2000)
    assert L.gq_atomic_peak(6, 1, 32, 1, buf, 1 << 20, sink, None) == gq.GQ_ERR_INVALID
    assert L.gq_atomic_peak(gq.GQ_PEAK_SPREAD_FAA, 1, 32, 1, buf, 16 * 512 - 1, sink, None) == gq.GQ_ERR_INVALID
    assert L.gq_atomic_peak(gq.GQ_PEAK_PACKED_FAA, 1, 32, 1, buf, 16 * 16 - 1, sink, None) == gq.GQ_ERR_INVALID
    assert L.gq_atomic_peak(gq.GQ_PEAK_SAME_ADDR_FAA, 1, 33, 1, buf, 64, sink, None) == gq.GQ_ERR_INVALID


def test_wavefaa_probe_arguments_validated():
    L = gq.load()
    p = ctypes.c_void_p(0x1000)   # never dereferenced: every call below fails validation first
    for width in (0, 3, 64):
        assert L.gq_wavefaa_probe(p, 64, width, p, p, None) == gq.GQ_ERR_INVALID
    assert L.gq_wavefaa_probe(p, 0, 32, p, p, None) == gq.GQ_ERR_INVALID
    assert L.gq_wavefaa_probe(None, 64, 32, p, p, None) == gq.GQ_ERR_INVALID


def test_run_multi_arguments_validated():
    L = gq.load()
    views = ctypes.c_void_p(0x1000)   # never dereferenced: every call below fails validation first
    good = dict(nqueues=4, threads_per_queue=64, producers_per_queue=32, block=256, blocks=0, kind=gq.KINDS["lfq"],
                elem_bytes=8, reserved=0, ops_per_queue=1000, d_counts=0x2000)
    bad = [dict(block=512), dict(block=0), dict(block=48), dict(threads_per_queue=48),
           dict(producers_per_queue=65), dict(kind=3), dict(elem_bytes=2), dict(nqueues=0), dict(d_counts=None)]
    for change in bad:
        a = gq.gq_multi_args(**dict(good, **change))
        assert L.gq_run_multi(views, ctypes.byref(a), None) == gq.GQ_ERR_INVALID, change


def test_run_rejects_null_arguments():
    L = gq.load()
    a = gq.gq_run_args(gq.GQ_RUN_PAIRS, 256, 256, 2, 0, 0, 0, None, None, None, None, None, 0x1000, None)
    assert L.gq_run(None, ctypes.byref(a), None) == gq.GQ_ERR_INVALID
    a.d_counts = None
    assert L.gq_run(ctypes.c_void_p(0x1000), ctypes.byref(a), None) == gq.GQ_ERR_INVALID


def test_run_rejects_bad_launch_shape():
    L = gq.load()
    h = ctypes.c_void_p(0x1000)   # never dereferenced: the launch shape is checked first
    for block, threads, ops in [(512, 256, 2), (48, 256, 2), (0, 256, 2), (256, 0, 2), (256, 256, 3)]:
        a = gq.gq_run_args(gq.GQ_RUN_PAIRS, threads, block, ops, 0, 0, 0, None, None, None, None, None, 0x2000, None)
        assert L.gq_run(h, ctypes.byref(a), None) == gq.GQ_ERR_INVALID, (block, threads, ops)


def test_binding_checks_buffers_before_the_call():
    # host tensors, undersized outputs and short counters never reach the C ABI
    import torch
    items = torch.zeros(16, dtype=torch.int64)
    with pytest.raises(gq.GqError) as ei:
        gq.gq_fifo_static_roundtrip(items, items, items[:1])
    assert ei.value.status == gq.GQ_ERR_INVALID and "CUDA" in str(ei.value)

    class FakeCuda:
        """Stands in for a CUDA tensor of the given size (no GPU here)."""
        is_cuda = True

        def __init__(self, n, es=8):
            self.n, self.es = n, es

        def numel(self):
            return self.n

        def element_size(self):
            return self.es

        def is_contiguous(self):
            return True

        def data_ptr(self):
            return 0

    with pytest.raises(gq.GqError, match="out"):
        gq.gq_fifo_static_roundtrip(FakeCuda(16), FakeCuda(8), FakeCuda(1))
    with pytest.raises(gq.GqError, match="num_out"):
        gq.gq_fifo_static_roundtrip(FakeCuda(16), FakeCuda(16), FakeCuda(1, 4))
    with pytest.raises(gq.GqError, match="items"):
        gq.gq_fifo_static_roundtrip(FakeCuda(16, 4), FakeCuda(16), FakeCuda(1), n=16)
