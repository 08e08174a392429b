"""G-WFQ-YMC specifics on the GPU against the oracle (run with -m gpu): the
slow paths (patience 0), the cell-pool bound, the reserved payload codes, and
the reset that clears only the cells an episode used."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2606_01693_gb300 as gq
import synth

from gpu_util import DEV, drain, make_queue, run_log, u64

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,p", [(1, 0.5), (2, 0.35), (3, 0.65)])
def test_slow_path_sequential_bit_exact(seed, p):
    kinds, vals = synth.random_op_list(seed, 3000, p)
    vals = vals % np.uint64(1 << 62)
    q = make_queue("ymc", 1 << 18, 8, max_threads=4, patience_enq=0, patience_deq=0)
    dk = torch.from_numpy(kinds).to(DEV)
    dv = torch.from_numpy(vals.view(np.int64)).to(DEV)
    ds = torch.zeros(len(kinds), dtype=torch.int8, device=DEV)
    do = torch.zeros(len(kinds), dtype=torch.int64, device=DEV)
    gq.gq_run_sequence(q.handle, dk, dv, ds, do)
    assert q.sync_status() == 0
    want_s, want_o, final = oracle.seqfifo_run(0, kinds, vals)
    assert (ds.cpu().numpy() == want_s).all()
    assert (u64(do) == want_o).all()
    assert (drain(q, len(kinds)) == final).all()


@pytest.mark.parametrize("patience", [0, 1, 10])
def test_concurrent_mixed_slow_and_fast(patience):
    T, K = 1 << 12, 50
    sched = synth.mixed_schedule_bits(31, T, K)
    q = make_queue("ymc", 1 << 22, 8, max_threads=T, patience_enq=patience, patience_deq=patience)
    r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched)
    left = drain(q, T * K)
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left)
    assert rep["violations"] == 0, str(rep)
    assert r["counts"][gq.GQ_CNT_ERRORS] == 0


@pytest.mark.parametrize("patience", [0, 2])
def test_tiny_histories_slow(patience):
    rng = np.random.default_rng(7 + patience)
    for trial in range(50):
        T = int(rng.integers(2, 7))
        K = max(1, min(4, 24 // T))
        sched = synth.mixed_schedule_bits(3000 + trial, T, K)
        q = make_queue("ymc", 1 << 12, 8, max_threads=32, patience_enq=patience, patience_deq=patience)
        r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched, block=32, timestamps=True,
                    delay_ns=int(rng.integers(0, 4000)))
        m = r["kind"].reshape(-1) != 255
        res = oracle.linearizable(r["kind"].reshape(-1)[m], r["val"].reshape(-1)[m], r["status"].reshape(-1)[m],
                                  r["call"].reshape(-1)[m], r["end"].reshape(-1)[m], cap=0)
        assert res == 1, (trial, r)
        q.close()


def test_pool_exhaustion_is_reported_not_faulted():
    q = make_queue("ymc", 64, 8, max_threads=256)
    items = torch.arange(1, 1001, dtype=torch.int64, device=DEV)
    st = torch.zeros(1000, dtype=torch.int8, device=DEV)
    ok = torch.zeros(1, dtype=torch.int64, device=DEV)
    q.enqueue(items, st, ok)
    assert q.sync_status() == gq.GQ_ERR_POOL_EXHAUSTED
    s = st.cpu().numpy()
    assert int(ok.item()) <= 64 and (s == gq.GQ_ERR_POOL_EXHAUSTED).sum() >= 1000 - 64
    q.reset()
    q.enqueue(items[:10], st[:10], ok)
    assert q.sync_status() == 0 and int(ok.item()) == 10


def test_reserved_payloads_rejected():
    q = make_queue("ymc", 1 << 10, 8, max_threads=256)
    items = torch.tensor([5, -1, -2, 7], dtype=torch.int64, device=DEV)   # 2^64-1 and 2^64-2 are reserved
    st = torch.zeros(4, dtype=torch.int8, device=DEV)
    ok = torch.zeros(1, dtype=torch.int64, device=DEV)
    q.enqueue(items, st, ok)
    assert q.sync_status() == 0
    assert st.cpu().tolist() == [0, gq.GQ_ERR_RESERVED_VALUE, gq.GQ_ERR_RESERVED_VALUE, 0]
    out = torch.zeros(4, dtype=torch.int64, device=DEV)
    q.dequeue(out, None, ok)
    assert q.sync_status() == 0
    assert sorted(out[: int(ok.item())].cpu().tolist()) == [5, 7]


@pytest.mark.parametrize("T", [1 << 12, 1 << 14])
def test_slow_dequeues_on_an_empty_heavy_split(T):
    # 90 % consumers with patience 0: the queue is empty most of the time, T
    # runs past the cells of published dequeue requests, and their candidate
    # searches walk more than 2^16 cells before they reach an empty cell
    q = make_queue("ymc", 1 << 26, 8, max_threads=T, patience_enq=0, patience_deq=0)
    P = T // 10
    r = run_log(q, gq.GQ_RUN_SPLIT, T, producers=P, total_ops=24 * T)
    left = drain(q, 24 * T)
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left)
    assert rep["violations"] == 0, str(rep)
    assert r["counts"][gq.GQ_CNT_ERRORS] == 0
    assert rep["deq_empty"] > 0


class _RingView(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("head", "tail", "threshold", "slots", "rec", "owner", "helpc",
                                                "slow_pending")]


class _DevView(ctypes.Structure):
    """Mirror of gq_dev (include/gq.h), to find the pool inside a caller-owned workspace."""
    _fields_ = ([(n, ctypes.c_uint32) for n in ("kind", "elem_bytes", "log2n", "cycle_bits", "max_threads",
                                                 "patience_enq", "patience_deq", "help_delay", "batch_width",
                                                 "ring_order", "backoff_ns", "due_wait", "patience_stretch",
                                                 "reserved1")]
                + [(n, ctypes.c_uint64) for n in ("capacity", "slot_mask", "cycle_mask", "cycle_half", "thr_reset")]
                + [("aq", _RingView), ("fq", _RingView)]
                + [(n, ctypes.c_void_p) for n in ("data", "err", "scratch", "ymc_tail", "ymc_head", "cell_val",
                                                   "cell_enq", "cell_deq", "ymc_rec", "ymc_hw")])


def test_reset_clears_every_cell_an_episode_touched():
    """gq_reset clears only the cells used since the previous reset: those below
    T and H and those the slow dequeues' candidate searches reached (the search
    mark).  After episodes whose searches run past T and H (90 % consumers,
    patience 0), every cell of the pool is clear again, and the reused pool
    gives runs that pass the run-log checks."""
    T, cap = 1 << 12, 1 << 22
    q = gq.Queue("ymc", cap, 8, max_threads=T, use_torch_memory=True, patience_enq=0, patience_deq=0)
    assert ctypes.sizeof(_DevView) <= gq.GQ_VIEW_BYTES
    view = _DevView()
    assert gq.load().gq_device_view(q.handle, ctypes.byref(view)) == 0
    assert view.capacity == cap
    base = (q._ws.data_ptr() + 255) // 256 * 256
    ws = q._ws[base - q._ws.data_ptr():]
    u64view = lambda ptr, n: ws[ptr - base: ptr - base + 8 * n].view(torch.int64)   # noqa: E731
    pairs = u64view(view.cell_val, 2 * (cap + 1)).view(cap + 1, 2)
    enq = u64view(view.cell_enq, cap + 1)
    ctl = lambda ptr: int(u64view(ptr, 1).item()) & ((1 << 64) - 1)   # noqa: E731
    P = T // 10
    for episode in range(3):
        r = run_log(q, gq.GQ_RUN_SPLIT, T, producers=P, total_ops=24 * T)
        left = drain(q, 24 * T)
        rep = oracle.check_log(r["kind"], r["status"], r["val"], left)
        assert rep["violations"] == 0, (episode, str(rep))
        torch.cuda.synchronize()
        t, h, hw = ctl(view.ymc_tail), ctl(view.ymc_head), ctl(view.ymc_hw)
        assert hw > 0 and max(t, h, hw + 1) <= cap + 1
        touched = (pairs[:, 0] != -1) | (pairs[:, 1] != 0) | (enq != 0)
        assert int(touched.sum().item()) > 0
        hi = int(torch.nonzero(touched).max().item())
        assert hi < max(t, h, hw + 1), (hi, t, h, hw)     # the bound covers every touched cell
        q.reset()
        torch.cuda.synchronize()
        assert ctl(view.ymc_hw) == 0 and ctl(view.ymc_tail) == 1
        assert bool((pairs[:, 0] == -1).all()) and bool((pairs[:, 1] == 0).all()) and bool((enq == 0).all())
    q.close()
