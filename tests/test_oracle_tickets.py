"""Pins for the oracle's ticket checker (CPU only).

The checker states three facts about recorded tickets (matching, distinct,
real-time order).  These tests pin it to logs whose verdict is known without
it: logs built by an independent FIFO simulation (every op linearized at a
point inside its interval, tickets drawn in linearization order) must pass,
and each planted mistake must be reported with its kind.
"""
import numpy as np
import pytest

import oracle

ENQ, DEQ = 1, 0


def fifo_log(seed, n_ops, p_enq=0.55, base=0, bits=64, jitter=30):
    """A concurrent-looking log from a sequential FIFO: op j is linearized at
    time 100 j; its interval is drawn around that point.  Enqueues take
    consecutive tickets base, base + 1, ... (mod 2^bits); a dequeue returns the
    oldest item and carries its ticket (the ring slot it was installed at)."""
    rng = np.random.default_rng(seed)
    mask = (1 << bits) - 1
    kind, status, val, tk, call, end = [], [], [], [], [], []
    fifo, nxt_tk, nxt_val = [], base, 1
    for j in range(n_ops):
        p = 100 * j
        c, e = p - int(rng.integers(0, jitter * 100)), p + int(rng.integers(0, jitter * 100))
        if rng.random() < p_enq:
            fifo.append((nxt_val, nxt_tk))
            kind.append(ENQ), status.append(0), val.append(nxt_val), tk.append(nxt_tk)
            nxt_val += 1
            nxt_tk = (nxt_tk + 1) & mask
        elif fifo:
            v, t = fifo.pop(0)
            kind.append(DEQ), status.append(0), val.append(v), tk.append(t)
        else:
            kind.append(DEQ), status.append(2), val.append(0), tk.append((1 << 64) - 1)
        call.append(c + 10 ** 6), end.append(e + 10 ** 6)
    return {"kind": np.array(kind, np.uint8), "status": np.array(status, np.int8),
            "val": np.array(val, np.uint64), "ticket": np.array(tk, np.uint64),
            "call": np.array(call, np.uint64), "end": np.array(end, np.uint64)}


def check(log, bits=64, stamps=True):
    return oracle.check_tickets(log["kind"], log["status"], log["val"], log["ticket"],
                                log["call"] if stamps else None, log["end"] if stamps else None, bits=bits)


@pytest.mark.parametrize("seed", range(6))
def test_fifo_logs_pass(seed):
    log = fifo_log(seed, 3000)
    rep = check(log)
    assert rep["violations"] == 0, rep
    assert rep["enq_ok"] == int(((log["kind"] == ENQ) & (log["status"] == 0)).sum())


@pytest.mark.parametrize("base,bits", [((1 << 64) - 700, 64), ((1 << 43) - 700, 43)])
def test_wrapping_tickets_pass(base, bits):
    rep = check(fifo_log(7, 3000, base=base, bits=bits), bits=bits)
    assert rep["violations"] == 0, rep


def test_43_bit_wrap_read_as_64_bits_fails():
    # the same log read without the wrap: the wrapped tickets look far smaller
    rep = check(fifo_log(8, 3000, base=(1 << 43) - 700, bits=43), bits=64)
    assert rep["violations"] > 0 and rep["first_kind"] in (10, 11)


def test_ticket_wider_than_counter():
    log = fifo_log(9, 200)
    j = int(np.flatnonzero((log["kind"] == ENQ) & (log["status"] == 0))[3])
    log["ticket"][j] |= np.uint64(1 << 50)
    rep = check(log, bits=43)
    assert rep["violations"] >= 1 and rep["first_kind"] == 7 and rep["first_index"] == j


def test_swapped_dequeue_tickets():
    log = fifo_log(10, 500)
    d = np.flatnonzero((log["kind"] == DEQ) & (log["status"] == 0))
    a, b = int(d[5]), int(d[40])
    log["ticket"][a], log["ticket"][b] = log["ticket"][b], log["ticket"][a]
    rep = check(log, stamps=False)
    assert rep["violations"] == 2 and rep["first_kind"] == 8


def test_dequeue_of_a_value_never_enqueued():
    log = fifo_log(11, 500)
    d = int(np.flatnonzero((log["kind"] == DEQ) & (log["status"] == 0))[7])
    log["val"][d] = np.uint64(10 ** 9)
    rep = check(log, stamps=False)
    assert rep["violations"] == 1 and rep["first_kind"] == 8 and rep["first_index"] == d


def test_duplicate_enqueue_ticket():
    log = fifo_log(12, 500, p_enq=0.9)
    e = np.flatnonzero((log["kind"] == ENQ) & (log["status"] == 0))
    log["ticket"][int(e[20])] = log["ticket"][int(e[19])]
    rep = check(log, stamps=False)
    assert rep["violations"] >= 1 and rep["first_kind"] == 9


def _log(rows):
    """rows: (kind, value, ticket, call, end), all successful."""
    k, v, t, c, e = zip(*rows)
    return {"kind": np.array(k, np.uint8), "status": np.zeros(len(rows), np.int8), "val": np.array(v, np.uint64),
            "ticket": np.array(t, np.uint64), "call": np.array(c, np.uint64), "end": np.array(e, np.uint64)}


def test_enqueue_tickets_against_real_time():
    # E1 returns before E2 is called, yet has the larger ticket; the dequeues overlap
    log = _log([(ENQ, 11, 1, 0, 1), (ENQ, 12, 0, 2, 3), (DEQ, 12, 0, 4, 10), (DEQ, 11, 1, 5, 9)])
    rep = check(log)
    assert rep["violations"] == 1 and rep["first_kind"] == 10 and rep["first_index"] == 1
    # the same tickets with overlapping enqueues are a valid history
    log["call"][1] = 0
    assert check(log)["violations"] == 0


def test_dequeue_tickets_against_real_time():
    log = _log([(ENQ, 11, 0, 0, 5), (ENQ, 12, 1, 1, 4), (DEQ, 12, 1, 6, 7), (DEQ, 11, 0, 8, 9)])
    rep = check(log)
    assert rep["violations"] == 1 and rep["first_kind"] == 11 and rep["first_index"] == 3
    log["end"][2] = 8                       # overlapping dequeues: valid
    assert check(log)["violations"] == 0


def test_failed_operations_are_ignored():
    log = _log([(ENQ, 11, 0, 0, 1), (DEQ, 11, 0, 2, 3)])
    log2 = {k: np.concatenate([v, v[:1]]) for k, v in log.items()}
    log2["status"][-1] = 1                  # a FULL enqueue with a stale ticket and value
    assert check(log2)["violations"] == 0
