"""Ticket checks on recorded GPU runs (run with -m gpu).

The run driver's recording kernel stores, for every successful operation, the
ticket it took effect at: the allocated-index ring position for G-LFQ and
G-WFQ (G-WFQ: a 43-bit Global counter value), the cell for G-WFQ-YMC.  The
oracle's ticket checker then requires that each dequeue carries its item's
enqueue ticket, that tickets are distinct, and that operations that do not
overlap in time take tickets in real-time order (Section III-B's linearization
at the ticket's slot; Section IV's device-side conformance checks).  The same
logs also go through the run-log invariant checks.
"""
import numpy as np
import pytest

import oracle
import paper_2606_01693_gb300 as gq
import synth

from gpu_util import drain, make_queue, run_log

pytestmark = pytest.mark.gpu

KINDS = list(gq.READY_KINDS)


def bits_of(kind):
    return 43 if kind == "wfq" else 64


def check_all(kind, r, left, **tok):
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left, **tok)
    assert rep["violations"] == 0, str(rep)
    tr = oracle.check_tickets(r["kind"], r["status"], r["val"], r["ticket"], r["call"], r["end"],
                              bits=bits_of(kind))
    assert tr["violations"] == 0, str(tr)
    ok = (r["status"] == 0) & (r["kind"] != 255)
    assert tr["enq_ok"] == int((ok & (r["kind"] == 1)).sum())
    assert tr["deq_ok"] == int((ok & (r["kind"] == 0)).sum())
    return tr


def pool(kind, cap, cells):
    return cells if kind == "ymc" else cap


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("T", [1 << 12, 1 << 16])
def test_mixed_tickets(kind, T):
    K = 64
    sched = synth.mixed_schedule_bits(3, T, K)
    q = make_queue(kind, pool(kind, 1 << 20, 1 << 23), 8, max_threads=T)
    r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched, timestamps=True, tickets=True)
    check_all(kind, r, drain(q, 1 << 20))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("frac", [0.1, 0.9])
def test_split_tickets_full_and_empty(kind, frac):
    T, total, cap = 1 << 16, 1 << 21, 1 << 12
    P = int(frac * T)
    q = make_queue(kind, pool(kind, cap, 1 << 22), 8, max_threads=T)
    r = run_log(q, gq.GQ_RUN_SPLIT, T, producers=P, total_ops=total, timestamps=True, tickets=True)
    check_all(kind, r, drain(q, total))


@pytest.mark.parametrize("kind", KINDS)
def test_pairs_one_block_tickets(kind):
    T, pairs = 256, 1000
    q = make_queue(kind, pool(kind, 1 << 10, 1 << 20), 4, max_threads=T)
    r = run_log(q, gq.GQ_RUN_PAIRS, T, 2 * pairs, timestamps=True, tickets=True)
    tr = check_all(kind, r, drain(q, 1 << 10), prod_shift=16, seq_mask=0xFFFF, seq_bias=0)
    assert tr["deq_ok"] == T * pairs


@pytest.mark.parametrize("kind", [k for k in KINDS if k != "lfq"])
def test_slow_path_tickets(kind):
    # patience 0: G-WFQ operations all go through SlowFAA and helping (D = 1);
    # G-WFQ-YMC makes one fast attempt, then publishes a request
    T, K = 1 << 12, 40
    sched = synth.mixed_schedule_bits(5, T, K)
    opt = dict(patience_enq=0, patience_deq=0)
    if kind == "wfq":
        opt["help_delay"] = 1
    q = make_queue(kind, pool(kind, 1 << 10, 1 << 22), 8, max_threads=T, **opt)
    r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched, timestamps=True, tickets=True, delay_ns=200)
    check_all(kind, r, drain(q, 1 << 10))


@pytest.mark.parametrize("kind", [k for k in KINDS if k != "ymc"])
def test_counter_wrap_tickets(kind):
    # counters start just below their wrap (2^64 for G-LFQ, 2^43 for G-WFQ's
    # Global words): tickets wrap during the run and are compared modulo 2^bits
    T, K, cap = 1 << 12, 64, 1 << 10
    start = (1 << 64) - (1 << 16) if kind == "lfq" else (1 << 43) - (1 << 16)
    sched = synth.mixed_schedule_bits(6, T, K)
    q = make_queue(kind, cap, 8, max_threads=T, start_ticket=start)
    r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=sched, timestamps=True, tickets=True)
    check_all(kind, r, drain(q, cap))
    ok = r["status"] == 0
    t = r["ticket"][ok]
    # some tickets were taken before the wrap and some after it
    assert (t >= np.uint64(start)).any() and (t < np.uint64(1 << 20)).any()
