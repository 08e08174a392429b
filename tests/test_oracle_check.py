"""Pins for the oracle's large-run invariant checker (CPU only).

Clean logs come from an independent Python simulation of a sequential FIFO
driven by an interleaving of T logical threads; planted mistakes (duplicated,
lost, reordered or overtaking tokens) must each be reported.
"""
import random
from collections import deque

import numpy as np
import pytest

import oracle
import synth


def simulate(T, K, seed, cap=0):
    rng = random.Random(seed)
    bits = synth.mixed_schedule_bits(seed, T, K)
    is_enq = synth.schedule_is_enq(bits, T, K)
    kind = np.where(is_enq.T, 1, 0).astype(np.uint8)      # op-major (K, T)
    status = np.zeros((K, T), np.int8)
    val = np.zeros((K, T), np.uint64)
    nxt = [0] * T
    seq = [0] * T
    q = deque()
    live = list(range(T))
    while live:
        t = rng.choice(live)
        i = nxt[t]
        if kind[i, t] == 1:
            tok = (t << 32) | (seq[t] + 1)
            seq[t] += 1
            val[i, t] = tok
            if cap and len(q) >= cap:
                status[i, t] = 1
            else:
                q.append(tok)
        else:
            if q:
                val[i, t] = q.popleft()
            else:
                status[i, t] = 2
        nxt[t] += 1
        if nxt[t] == K:
            live.remove(t)
    return kind, status, val, np.array(list(q), np.uint64)


@pytest.mark.parametrize("cap", [0, 8])
def test_clean_log_passes(cap):
    kind, status, val, drained = simulate(16, 40, 3, cap)
    rep = oracle.check_log(kind, status, val, drained)
    assert rep["violations"] == 0, rep
    assert rep["enq_ok"] + rep["enq_full"] == int((kind == 1).sum())
    assert rep["deq_ok"] + rep["deq_empty"] == int((kind == 0).sum())
    assert rep["enq_ok"] == rep["deq_ok"] + len(drained)
    if cap:
        assert rep["enq_full"] > 0


def _deq_positions(kind, status):
    return [tuple(x) for x in np.argwhere((kind == 0) & (status == 0))]


def test_duplicate_reported():
    kind, status, val, drained = simulate(16, 40, 4)
    pos = _deq_positions(kind, status)
    a, b = pos[3], pos[10]
    val[b] = val[a]
    rep = oracle.check_log(kind, status, val, drained)
    assert rep["violations"] > 0 and rep["first_kind"] == 1


def test_lost_item_reported():
    kind, status, val, drained = simulate(16, 40, 5)
    pos = _deq_positions(kind, status)
    status[pos[7]] = 2
    rep = oracle.check_log(kind, status, val, drained)
    assert rep["violations"] > 0 and rep["first_kind"] == 1


def test_reorder_within_consumer_reported():
    # find a consumer that dequeued two tokens of the same producer, swap them
    for seed in range(6, 40):
        kind, status, val, drained = simulate(4, 60, seed)
        for t in range(4):
            rows = [i for i in range(60) if kind[i, t] == 0 and status[i, t] == 0]
            by_p = {}
            for i in rows:
                by_p.setdefault(int(val[i, t]) >> 32, []).append(i)
            for p, lst in by_p.items():
                if len(lst) >= 2:
                    i1, i2 = lst[0], lst[1]
                    val[i1, t], val[i2, t] = val[i2, t], val[i1, t]
                    rep = oracle.check_log(kind, status, val, drained)
                    assert rep["violations"] > 0 and rep["first_kind"] == 2
                    return
    pytest.fail("no consumer with two tokens of one producer")


def test_overtaking_and_drain_order_reported():
    kind, status, val, drained = simulate(8, 60, 11)
    # overtaking: pretend the oldest dequeued token of some producer is still in the queue
    pos = _deq_positions(kind, status)
    tok = int(val[pos[0]])
    p = tok >> 32
    later = [int(val[x]) for x in pos if int(val[x]) >> 32 == p and int(val[x]) != tok]
    if later:
        bad_drained = np.concatenate([drained, np.array([tok], np.uint64)])
        status2 = status.copy()
        status2[pos[0]] = 2
        rep = oracle.check_log(kind, status2, val, bad_drained)
        assert rep["violations"] > 0 and rep["first_kind"] == 3
    # drain order: reverse two drained tokens of one producer
    d = np.array([(1 << 32) | 1, (1 << 32) | 2], np.uint64)
    K, T = 1, 2
    kind2 = np.array([[1, 1]], np.uint8)
    st2 = np.zeros((1, 2), np.int8)
    v2 = np.array([[(1 << 32) | 1, (1 << 32) | 2]], np.uint64)
    assert oracle.check_log(kind2, st2, v2, d)["violations"] == 0
    rep = oracle.check_log(kind2, st2, v2, d[::-1].copy())
    assert rep["violations"] > 0 and rep["first_kind"] == 4


def test_bad_status_and_token_reported():
    kind, status, val, drained = simulate(4, 20, 12)
    pos = _deq_positions(kind, status)
    s2 = status.copy(); s2[pos[0]] = 1                 # FULL on a dequeue
    assert oracle.check_log(kind, s2, val, drained)["first_kind"] == 6
    v2 = val.copy(); v2[pos[0]] = 0                     # seq field 0 decodes to no token
    rep = oracle.check_log(kind, status, v2, drained)
    assert rep["violations"] > 0
