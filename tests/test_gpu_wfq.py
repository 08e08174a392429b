"""G-WFQ slow path on the GPU against the oracle (run with -m gpu).

Patience 0 sends every operation through the cooperative slow path
(Algorithm 2: SlowFAA, TryEnqSlow / TryDeqSlow, phase-2 helping, Enq-bit
finalisation); help delay D = 1 makes every operation inspect and help a peer
record.  Results must still be exactly the sequential FIFO's (one thread) or
pass the linearizability and run-log checks (many threads).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_01693_gb300 as gq
import synth

from gpu_util import DEV, drain, make_queue, run_log, u64

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cap,seed", [(2, 1), (4, 2), (64, 3)])
def test_slow_path_sequential_bit_exact(cap, seed):
    kinds, vals = synth.random_op_list(seed, 3000, 0.5)
    q = make_queue("wfq", cap, 8, max_threads=1, help_delay=1, patience_enq=0, patience_deq=0)
    dk = torch.from_numpy(kinds).to(DEV)
    dv = torch.from_numpy(vals.view(np.int64)).to(DEV)
    ds = torch.zeros(len(kinds), dtype=torch.int8, device=DEV)
    do = torch.zeros(len(kinds), dtype=torch.int64, device=DEV)
    gq.gq_run_sequence(q.handle, dk, dv, ds, do)
    assert q.sync_status() == 0
    want_s, want_o, final = oracle.seqfifo_run(cap, kinds, vals)
    assert (ds.cpu().numpy() == want_s).all()
    assert (u64(do) == want_o).all()
    assert (drain(q, cap) == final).all()
    st = q.stats()
    # every ring operation went slow: each queue op is two ring ops
    assert st["slow_requests"] >= len(kinds)


@pytest.mark.parametrize("patience,stretch", [(0, 0), (1, 1), (1, 0)])
@pytest.mark.parametrize("help_delay", [1, 64])
def test_slow_path_concurrent_mixed(patience, stretch, help_delay):
    # stretch 0 = the default patience stretch (fast attempts go on while
    # requests of the ring are pending), 1 = off
    T, K = 1 << 12, 40
    sched = synth.mixed_schedule_bits(17, T, K)
    q = make_queue("wfq", 1 << 10, 8, max_threads=T, help_delay=help_delay,
                   patience_enq=patience, patience_deq=patience, patience_stretch=stretch)
    r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched)
    left = drain(q, 1 << 10)
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left)
    assert rep["violations"] == 0, str(rep)
    assert r["counts"][gq.GQ_CNT_ERRORS] == 0
    st = q.stats()
    assert st["slow_requests"] > 0
    if help_delay == 1 and patience == 0:
        assert st["helps"] > 0


@pytest.mark.parametrize("frac", [0.1, 0.9])
def test_slow_path_split_full_and_empty(frac):
    T, total, cap = 1 << 12, 200000, 1 << 8
    P = int(frac * T)
    q = make_queue("wfq", cap, 8, max_threads=T, patience_enq=0, patience_deq=0, help_delay=8)
    r = run_log(q, gq.GQ_RUN_SPLIT, T, producers=P, total_ops=total)
    left = drain(q, cap)
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left)
    assert rep["violations"] == 0, str(rep)
    assert rep["enq_full"] > 0 if frac == 0.9 else rep["deq_empty"] > 0


@pytest.mark.parametrize("patience", [0, 2])
def test_slow_path_tiny_histories(patience):
    rng = np.random.default_rng(100 + patience)
    for trial in range(50):
        T = int(rng.integers(2, 7))
        K = max(1, min(4, 24 // T))
        sched = synth.mixed_schedule_bits(2000 + trial, T, K)
        cap = int(rng.choice([2, 4]))
        q = make_queue("wfq", cap, 8, max_threads=32, help_delay=1, patience_enq=patience, patience_deq=patience)
        r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched, block=32, timestamps=True,
                    delay_ns=int(rng.integers(0, 4000)))
        m = r["kind"].reshape(-1) != 255
        res = oracle.linearizable(r["kind"].reshape(-1)[m], r["val"].reshape(-1)[m], r["status"].reshape(-1)[m],
                                  r["call"].reshape(-1)[m], r["end"].reshape(-1)[m], cap=cap)
        assert res == 1, (trial, r)
        q.close()


@pytest.mark.parametrize("stretch", [1, 4, 64])
@pytest.mark.parametrize("frac", [0.1, 0.5, 0.9])
def test_patience_stretch_split_oversubscribed(stretch, frac):
    # more threads than slots, small patience: operations run out of patience
    # while requests are already pending, the case the stretch is for; every
    # stretch setting must keep the run log valid and leave no request pending
    T, total, cap = 1 << 13, 300000, 1 << 8
    q = make_queue("wfq", cap, 8, max_threads=T, patience_enq=2, patience_deq=4, help_delay=16,
                   patience_stretch=stretch)
    r = run_log(q, gq.GQ_RUN_SPLIT, T, producers=int(frac * T), total_ops=total)
    left = drain(q, cap)
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left)
    assert rep["violations"] == 0, str(rep)
    assert r["counts"][gq.GQ_CNT_ERRORS] == 0
    st = q.stats()
    assert st["slow_requests"] > 0
    assert st["aq_slow_pending"] == 0 and st["fq_slow_pending"] == 0, st


def test_delay_injection_many_threads():
    # delayed threads stall mid-run; helpers must finish their published requests
    T, K = 1 << 11, 30
    sched = synth.mixed_schedule_bits(23, T, K)
    q = make_queue("wfq", 1 << 9, 8, max_threads=T, patience_enq=1, patience_deq=1, help_delay=2)
    r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched, delay_ns=20000)
    left = drain(q, 1 << 9)
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left)
    assert rep["violations"] == 0, str(rep)


def test_bulk_throughput_shape_with_slow_path_counts():
    # the benchmark configuration: slow-path entries must stay rare with default patience
    T, K = 1 << 18, 100
    sched = synth.mixed_schedule_bits(0, T, K)
    q = make_queue("wfq", 1 << 20, 8, max_threads=T)
    r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched)
    left = drain(q, 1 << 20)
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left)
    assert rep["violations"] == 0, str(rep)
    st = q.stats()
    assert st["slow_requests"] < 0.01 * T * K, st


def _delta(a, b):
    return (b - a) % (1 << 43)          # Counter fields of the Global words are 43 bits


@pytest.mark.parametrize("help_delay,delay_ns", [(1, 0), (64, 0), (2, 20000)])
def test_slow_rounds_account_for_every_head_ticket(help_delay, delay_ns):
    # Algorithm 2: a successful SlowFAA round advances the Global Counter by
    # exactly one.  With patience 0 no fast-path fetch-add runs, so the two Head
    # words move only by slow rounds (catch-up raises Tail words only): the
    # Head tickets issued equal the slow rounds counted on the head side, and
    # the Tail tickets issued are at least the tail-side rounds.
    T, K = 1 << 11, 30
    sched = synth.mixed_schedule_bits(29, T, K)
    q = make_queue("wfq", 1 << 9, 8, max_threads=T, patience_enq=0, patience_deq=0, help_delay=help_delay)
    s0 = q.stats()
    r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched, delay_ns=delay_ns)
    s1 = q.stats()
    assert r["counts"][gq.GQ_CNT_ERRORS] == 0
    heads = _delta(s0["aq_head"], s1["aq_head"]) + _delta(s0["fq_head"], s1["fq_head"])
    tails = _delta(s0["aq_tail"], s1["aq_tail"]) + _delta(s0["fq_tail"], s1["fq_tail"])
    assert s1["slow_rounds_head"] > 0 and heads == s1["slow_rounds_head"], (s0, s1)
    assert s1["slow_rounds_tail"] > 0 and tails >= s1["slow_rounds_tail"], (s0, s1)
    # every operation went slow on both of its rings
    ok = int(r["counts"][gq.GQ_CNT_ENQ_OK] + r["counts"][gq.GQ_CNT_DEQ_OK])
    assert s1["slow_requests"] >= 2 * ok
    # wait-freedom, empirically: no helper came near the hard iteration cap;
    # with all 2^11 threads on the slow path one helper needed at most about
    # 31 k iterations (k = threads) for one request
    print("max SlowFAA iterations of one helper on one request:", s1["max_help_iterations"])
    assert 0 < s1["max_help_iterations"] <= 256 * T + (1 << 16)


def test_fast_path_tickets_outnumber_slow_rounds():
    # default patience: fetch-adds issue most tickets, SlowFAA rounds are a subset
    T, K = 1 << 16, 64
    sched = synth.mixed_schedule_bits(31, T, K)
    q = make_queue("wfq", 1 << 12, 8, max_threads=T)
    s0 = q.stats()
    r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched, record=False)
    s1 = q.stats()
    heads = _delta(s0["aq_head"], s1["aq_head"]) + _delta(s0["fq_head"], s1["fq_head"])
    tails = _delta(s0["aq_tail"], s1["aq_tail"]) + _delta(s0["fq_tail"], s1["fq_tail"])
    # a successful operation takes at least one Head ticket (fq for an enqueue, aq for a dequeue)
    assert heads >= int(r["counts"][gq.GQ_CNT_ENQ_OK] + r["counts"][gq.GQ_CNT_DEQ_OK])
    assert s1["slow_rounds_head"] <= heads and s1["slow_rounds_tail"] <= tails
