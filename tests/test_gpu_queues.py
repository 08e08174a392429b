"""GPU parity tests: the CUDA queues against the CPU oracle (run with -m gpu).

Every test calls the CUDA path through the C ABI (libgq.so) and checks the
results with the oracle, which shares no code with it:
  * sequential bit-exactness against the FIFO specification (FULL at exactly n
    items, EMPTY at exactly 0, ring and cycle-tag wrap-around);
  * the one-block pairs workload (256 threads x 1000 enqueue-then-dequeue pairs,
    capacity 2^10, 32-bit tokens): zero EMPTY, zero FULL, exactly once,
    per-producer order;
  * the 50/50 interleaved workload up to 2^20 threads x 100 ops at capacity
    2^20, its enqueue-only-then-dequeue-only phase form, and the imbalanced
    producer/consumer workload (2^18 threads, 10^7 ops,
    capacity 2^16) with the run-log invariant checks;
  * linearizability of tiny recorded histories (Wing & Gong);
  * the host batch API (exactly once through gq_enqueue_batch/gq_dequeue_batch).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_01693_gb300 as gq
import synth

from gpu_util import DEV, drain, make_queue, run_log, u64

pytestmark = pytest.mark.gpu

KINDS = list(gq.READY_KINDS)


def qcap(kind, cap, pool=1 << 22):
    """(capacity argument, oracle capacity): G-WFQ-YMC is unbounded (never FULL);
    its capacity argument is the cell pool, sized for the run's tickets."""
    return (pool, 0) if kind == "ymc" else (cap, cap)


def _seq_ops(seed, n, cap, p_enq):
    kinds, vals = synth.random_op_list(seed, n, p_enq)
    return kinds, vals


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("cap,cycle_bits,seed,p", [(2, 0, 1, 0.5), (2, 3, 2, 0.55), (4, 3, 3, 0.5),
                                                  (16, 0, 4, 0.6), (16, 3, 5, 0.45), (1024, 0, 6, 0.5)])
@pytest.mark.parametrize("elem", [4, 8])
def test_sequential_bit_exact(kind, cap, cycle_bits, seed, p, elem):
    n = 4000
    kinds, vals = _seq_ops(seed, n, cap, p)
    if elem == 4:
        vals = vals & np.uint64(0xFFFFFFFF)
    # one record and D = 1 keep G-WFQ's soundness bound R > Dk/n + 6 within small cycle tags
    extra = dict(max_threads=1, help_delay=1) if kind == "wfq" else dict(max_threads=64)
    if kind != "ymc":
        extra["cycle_bits"] = cycle_bits
    qc, ocap = qcap(kind, cap, pool=1 << 16)
    q = make_queue(kind, qc, elem, **extra)
    dk = torch.from_numpy(kinds).to(DEV)
    dv = torch.from_numpy(vals.view(np.int64)).to(DEV)
    ds = torch.zeros(n, dtype=torch.int8, device=DEV)
    do = torch.zeros(n, dtype=torch.int64, device=DEV)
    gq.gq_run_sequence(q.handle, dk, dv, ds, do)
    assert q.sync_status() == 0
    want_s, want_o, final = oracle.seqfifo_run(ocap, kinds, vals)
    got_s = ds.cpu().numpy()
    got_o = u64(do)
    assert (got_s == want_s).all(), np.flatnonzero(got_s != want_s)[:5]
    assert (got_o == want_o).all()
    assert (drain(q, max(cap, len(final))) == final).all()
    # the spec's boundaries were crossed: EMPTY at 0 items, and FULL at n items for small rings
    assert (want_s == 2).any()
    if cap <= 16 and ocap:
        assert (want_s == 1).any()


@pytest.mark.parametrize("kind", [k for k in KINDS if k != "ymc"])
def test_sequential_counter_wrap(kind):
    # counters start 3 * 2n tickets before 2^64 (G-LFQ) so ticket arithmetic wraps mid-run
    cap = 8
    start = (1 << 64) - 4 * 2 * cap if kind == "lfq" else (1 << 43) - 4 * 2 * cap
    kinds, vals = _seq_ops(11, 3000, cap, 0.5)
    q = make_queue(kind, cap, 8, max_threads=64, start_ticket=start)
    dk = torch.from_numpy(kinds).to(DEV)
    dv = torch.from_numpy(vals.view(np.int64)).to(DEV)
    ds = torch.zeros(len(kinds), dtype=torch.int8, device=DEV)
    do = torch.zeros(len(kinds), dtype=torch.int64, device=DEV)
    gq.gq_run_sequence(q.handle, dk, dv, ds, do)
    assert q.sync_status() == 0
    want_s, want_o, final = oracle.seqfifo_run(cap, kinds, vals)
    assert (ds.cpu().numpy() == want_s).all()
    assert (u64(do) == want_o).all()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("width", [32, 1])
def test_pairs_one_block(kind, width):
    # 1 block x 256 threads, 1000 enqueue-then-dequeue pairs each, capacity 2^10, u32 tokens (t << 16) | seq
    T, pairs = 256, 1000
    qc, _ = qcap(kind, 1 << 10, pool=1 << 20)
    q = make_queue(kind, qc, 4, max_threads=T, batch_width=width)
    r = run_log(q, gq.GQ_RUN_PAIRS, T, 2 * pairs)
    c = r["counts"]
    assert c[gq.GQ_CNT_ENQ_OK] == T * pairs and c[gq.GQ_CNT_DEQ_OK] == T * pairs
    assert c[gq.GQ_CNT_ENQ_FULL] == 0 and c[gq.GQ_CNT_DEQ_EMPTY] == 0   # balanced closed form
    assert c[gq.GQ_CNT_ERRORS] == 0
    assert c[gq.GQ_CNT_SUM_ENQ] == c[gq.GQ_CNT_SUM_DEQ]
    left = drain(q, 1 << 10)
    assert len(left) == 0
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left, prod_shift=16, seq_mask=0xFFFF, seq_bias=0)
    assert rep["violations"] == 0, str(rep)
    assert rep["deq_ok"] == T * pairs


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("T", [1 << 10, 1 << 14])
def test_mixed_interleaved(kind, T):
    K = 100
    sched = synth.mixed_schedule_bits(0, T, K)
    qc, _ = qcap(kind, 1 << 20, pool=1 << 23)
    q = make_queue(kind, qc, 8, max_threads=T)
    r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched)
    left = drain(q, 1 << 20)
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left)
    assert rep["violations"] == 0, str(rep)
    assert rep["enq_full"] == 0
    assert rep["enq_ok"] == int(synth.schedule_is_enq(sched, T, K).sum())


@pytest.mark.parametrize("kind", KINDS)
def test_mixed_full_size(kind):
    # the largest configuration of the throughput sweep: 2^20 threads x 100 ops, capacity 2^20
    T, K = 1 << 20, 100
    sched = synth.mixed_schedule_bits(0, T, K)
    qc, _ = qcap(kind, 1 << 20, pool=1 << 27)
    q = make_queue(kind, qc, 8, max_threads=T)
    r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched)
    left = drain(q, 1 << 20)
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left)
    assert rep["violations"] == 0, str(rep)
    c = r["counts"]
    assert c[gq.GQ_CNT_ERRORS] == 0
    assert (int(c[gq.GQ_CNT_SUM_ENQ]) - int(c[gq.GQ_CNT_SUM_DEQ]) - int(left.sum(dtype=np.uint64))) % (1 << 64) == 0


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("frac", [0.1, 0.5, 0.9])
def test_split_producer_consumer(kind, frac):
    T, total, cap = 1 << 18, 10 ** 7, 1 << 16
    P = int(frac * T)
    qc, ocap = qcap(kind, cap, pool=1 << 25)
    q = make_queue(kind, qc, 8, max_threads=T)
    r = run_log(q, gq.GQ_RUN_SPLIT, T, producers=P, total_ops=total)
    left = drain(q, total)
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left)
    assert rep["violations"] == 0, str(rep)
    assert rep["enq_ok"] + rep["enq_full"] == int(synth.split_ops_per_thread(total, T)[:P].sum())
    if ocap:
        assert len(left) <= cap
    if frac == 0.9 and ocap:
        assert rep["enq_full"] > 0          # the bounded queue filled up
    if frac == 0.1:
        assert rep["deq_empty"] > 0


@pytest.mark.parametrize("kind", ["lfq", "wfq"])
@pytest.mark.parametrize("frac", [0.1, 0.9])
def test_split_with_due_install_wait(kind, frac):
    """The ring queues with the due-install wait on (a dequeuer re-reads a slot
    whose enqueuer is due before ruling it out): same checks as the plain run."""
    T, total, cap = 1 << 16, 1 << 21, 1 << 12
    P = int(frac * T)
    q = make_queue(kind, cap, 8, max_threads=T, due_wait=64)
    r = run_log(q, gq.GQ_RUN_SPLIT, T, producers=P, total_ops=total, tickets=True)
    left = drain(q, total)
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left)
    assert rep["violations"] == 0, str(rep)
    tr = oracle.check_tickets(r["kind"], r["status"], r["val"], r["ticket"], bits=43 if kind == "wfq" else 64)
    assert tr["violations"] == 0, str(tr)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("T", [1 << 10, 1 << 14, 1 << 20])
def test_enqueue_then_dequeue_phases(kind, T):
    """The sweep workload's phase form: every thread enqueues its share of
    min(2^20, 100 T) items, then (a second launch) every thread dequeues the same
    number.  All succeed, the queue ends empty, and the concatenated log passes the
    exactly-once and per-producer-order checks."""
    cap = 1 << 20
    target = min(cap, 100 * T)
    qc, _ = qcap(kind, cap, pool=1 << 22)
    q = make_queue(kind, qc, 8, max_threads=T)
    a = run_log(q, gq.GQ_RUN_SPLIT, T, producers=T, total_ops=target)
    b = run_log(q, gq.GQ_RUN_SPLIT, T, producers=0, total_ops=target)
    assert a["counts"][gq.GQ_CNT_ENQ_OK] == target and a["counts"][gq.GQ_CNT_ENQ_FULL] == 0
    assert b["counts"][gq.GQ_CNT_DEQ_OK] == target and b["counts"][gq.GQ_CNT_DEQ_EMPTY] == 0
    left = drain(q, 16)
    assert len(left) == 0
    rep = oracle.check_log(np.concatenate([a["kind"], b["kind"]]), np.concatenate([a["status"], b["status"]]),
                           np.concatenate([a["val"], b["val"]]), left)
    assert rep["violations"] == 0, str(rep)
    assert rep["enq_ok"] == rep["deq_ok"] == target


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("cap", [2, 4])
def test_tiny_histories_linearizable(kind, cap):
    rng = np.random.default_rng(cap)
    checked = 0
    for trial in range(60):
        T = int(rng.integers(2, 7))
        K = int(rng.integers(2, 5))
        if T * K > 24:
            K = 24 // T
        sched = synth.mixed_schedule_bits(1000 + trial, T, K)
        qc, ocap = qcap(kind, cap, pool=1 << 10)
        q = make_queue(kind, qc, 8, max_threads=64)
        r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched, block=32, timestamps=True,
                    delay_ns=int(rng.integers(0, 3000)))
        m = r["kind"].reshape(-1) != 255
        op = r["kind"].reshape(-1)[m]
        res = oracle.linearizable(op, r["val"].reshape(-1)[m], r["status"].reshape(-1)[m],
                                  r["call"].reshape(-1)[m], r["end"].reshape(-1)[m], cap=ocap)
        assert res == 1, (trial, r)
        checked += 1
        q.close()
    assert checked == 60


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("elem", [4, 8])
def test_batch_api_exactly_once(kind, elem):
    cap = 1 << 12
    qc, ocap = qcap(kind, cap, pool=1 << 16)
    q = make_queue(kind, qc, elem, max_threads=1 << 16)
    dt = torch.int32 if elem == 4 else torch.int64
    n = cap + 1000                                        # bounded rings: 1000 attempts must fail FULL
    items = torch.arange(1, n + 1, dtype=dt, device=DEV) * 7
    st = torch.zeros(n, dtype=torch.int8, device=DEV)
    ok = torch.zeros(1, dtype=torch.int64, device=DEV)
    q.enqueue(items, st, ok)
    assert q.sync_status() == 0
    s = st.cpu().numpy()
    if not ocap:
        cap = n                                           # unbounded: every enqueue succeeds
    assert int(ok.item()) == cap
    assert (s == 0).sum() == cap and (s == 1).sum() == n - cap
    out = torch.zeros(n, dtype=dt, device=DEV)
    st2 = torch.zeros(n, dtype=torch.int8, device=DEV)
    ok2 = torch.zeros(1, dtype=torch.int64, device=DEV)
    q.dequeue(out, st2, ok2)
    assert q.sync_status() == 0
    k = int(ok2.item())
    assert k == cap and (st2.cpu().numpy() == 2).sum() == n - cap
    got = np.sort(out[:k].cpu().numpy())
    want = np.sort(items.cpu().numpy()[s == 0])
    assert (got == want).all()


@pytest.mark.parametrize("kind", KINDS)
def test_caller_owned_workspace(kind):
    q = gq.Queue(kind, 1 << 10, 8, 1024, use_torch_memory=True)   # G-WFQ-YMC: 1024 pool cells
    assert gq.gq_info(q.handle)[1] is False
    items = torch.arange(100, dtype=torch.int64, device=DEV)
    q.enqueue(items)
    out = torch.zeros(100, dtype=torch.int64, device=DEV)
    ok = torch.zeros(1, dtype=torch.int64, device=DEV)
    q.dequeue(out, None, ok)
    assert q.sync_status() == 0
    assert int(ok.item()) == 100
    assert sorted(out.cpu().tolist()) == list(range(100))
    q.reset()
    q.dequeue(out, None, ok)
    assert q.sync_status() == 0 and int(ok.item()) == 0


def test_capped_run_captured_in_a_graph():
    # a G-LFQ run of 2^18 threads (1024 blocks) on a ring of capacity 2^16 is
    # launched with the residency cap (more threads than slots); made only
    # inside stream capture, it replays like an eager launch: every attempt is
    # counted once and what was enqueued and not dequeued is what remains
    T, total, cap = 1 << 18, 1 << 20, 1 << 16
    q = make_queue("lfq", cap, 8, max_threads=T)
    counts = torch.zeros(8, dtype=torch.int64, device=DEV)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        q.reset()
        counts.zero_()
        gq.gq_run(q.handle, gq.GQ_RUN_SPLIT, T, block=256, producers=T // 2, total_ops=total, counts=counts)
    for _ in range(3):
        g.replay()
        torch.cuda.synchronize()
        c = u64(counts)
        assert c[gq.GQ_CNT_ERRORS] == 0, c
        assert c[gq.GQ_CNT_ENQ_OK] + c[gq.GQ_CNT_ENQ_FULL] + c[gq.GQ_CNT_DEQ_OK] + c[gq.GQ_CNT_DEQ_EMPTY] == total
        assert c[gq.GQ_CNT_ENQ_OK] > 0 and c[gq.GQ_CNT_DEQ_OK] > 0
        left = drain(q, cap)
        assert len(left) == int(c[gq.GQ_CNT_ENQ_OK] - c[gq.GQ_CNT_DEQ_OK])
        assert (int(c[gq.GQ_CNT_SUM_ENQ]) - int(c[gq.GQ_CNT_SUM_DEQ])) % (1 << 64) == int(left.sum(dtype=np.uint64))
    assert q.sync_status() == 0


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("elem", [4, 8])
@pytest.mark.parametrize("shift", [0, 1])
def test_batch_api_tiles_tail_and_alignment(kind, elem, shift):
    """The dequeue batch's tiled path (several attempts per lane, values staged in
    shared memory and stored compacted) and its one-attempt-per-lane path (a tail
    shorter than a tile; a status buffer not aligned for the tile's status store:
    shift = 1 offsets items, outputs and statuses by one element) give the same
    exactly-once result."""
    n = (1 << 15) + 37
    qc, _ = qcap(kind, 1 << 16, pool=1 << 18)
    q = make_queue(kind, qc, elem, max_threads=1 << 16)
    dt = torch.int32 if elem == 4 else torch.int64
    base = torch.arange(1, n + 2, dtype=dt, device=DEV) * 3
    items = base[shift:shift + n]
    st_all = torch.full((n + 1,), -99, dtype=torch.int8, device=DEV)
    st = st_all[shift:shift + n]
    ok = torch.zeros(1, dtype=torch.int64, device=DEV)
    q.enqueue(items, st, ok)
    assert q.sync_status() == 0
    assert int(ok.item()) == n and (st.cpu().numpy() == 0).all()
    out_all = torch.zeros(n + 1, dtype=dt, device=DEV)
    out = out_all[shift:shift + n]
    st2_all = torch.full((n + 1,), -99, dtype=torch.int8, device=DEV)
    st2 = st2_all[shift:shift + n]
    ok2 = torch.zeros(1, dtype=torch.int64, device=DEV)
    q.dequeue(out, st2, ok2)
    assert q.sync_status() == 0
    assert int(ok2.item()) == n and (st2.cpu().numpy() == 0).all()
    assert (np.sort(out.cpu().numpy()) == np.sort(items.cpu().numpy())).all()
    q.dequeue(out[:64], st2[:64], ok2)                  # now empty
    assert q.sync_status() == 0
    assert int(ok2.item()) == 0 and (st2[:64].cpu().numpy() == 2).all()
