"""Pins for the oracle's sequential FIFO and mutex-deque baseline (CPU only).

The sequential FIFO is pinned to a hand-worked example (tests/golden), to closed
forms (n enqueues then n dequeues return the same order; FULL at exactly the
capacity, EMPTY at exactly zero) and to an independent list-based replay.
"""
import os
from collections import deque

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ST = {"OK": 0, "FULL": 1, "EMPTY": 2}


def _load_seqfifo_golden():
    kinds, vals, status, outs = [], [], [], []
    for line in open(os.path.join(GOLDEN, "seqfifo_cap3.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        f = line.split()
        kinds.append(1 if f[0] == "enq" else 0)
        vals.append(int(f[1]) if f[1] != "-" else 0)
        status.append(ST[f[2]])
        outs.append(int(f[3]) if len(f) > 3 else 0)
    return (np.array(kinds, np.uint8), np.array(vals, np.uint64), np.array(status, np.int8),
            np.array(outs, np.uint64))


def test_seqfifo_matches_hand_worked_example():
    kinds, vals, status, outs = _load_seqfifo_golden()
    s, o, final = oracle.seqfifo_run(3, kinds, vals)
    assert s.tolist() == status.tolist()
    assert o.tolist() == outs.tolist()
    assert len(final) == 0


@pytest.mark.parametrize("n", [1, 2, 7, 64])
def test_seqfifo_closed_form_fill_and_drain(n):
    vals = np.arange(1000, 1000 + n + 1, dtype=np.uint64)
    kinds = np.array([1] * (n + 1) + [0] * (n + 1), np.uint8)
    allv = np.concatenate([vals, np.zeros(n + 1, np.uint64)])
    s, o, final = oracle.seqfifo_run(n, kinds, allv)
    # FULL exactly at the (n+1)-th enqueue, EMPTY exactly at the (n+1)-th dequeue
    assert s[:n].tolist() == [0] * n and s[n] == 1
    assert s[n + 1: 2 * n + 1].tolist() == [0] * n and s[2 * n + 1] == 2
    assert o[n + 1: 2 * n + 1].tolist() == vals[:n].tolist()
    assert len(final) == 0


def _list_replay(cap, kinds, vals):
    q, st, out = [], [], []
    for k, v in zip(kinds.tolist(), vals.tolist()):
        if k == 1:
            if cap and len(q) >= cap:
                st.append(1); out.append(0)
            else:
                q.append(v); st.append(0); out.append(0)
        else:
            if not q:
                st.append(2); out.append(0)
            else:
                st.append(0); out.append(q.pop(0))
    return st, out, q


@pytest.mark.parametrize("cap,seed,p", [(0, 1, 0.5), (4, 2, 0.6), (16, 3, 0.55), (2, 4, 0.5)])
def test_seqfifo_matches_independent_replay(cap, seed, p):
    kinds, vals = synth.random_op_list(seed, 3000, p)
    s, o, final = oracle.seqfifo_run(cap, kinds, vals)
    st, out, q = _list_replay(cap, kinds, vals)
    assert s.tolist() == st
    assert o.tolist() == out
    assert final.tolist() == q


def test_mutex_pairs_closed_form():
    # Every thread enqueues before it dequeues, so the k-th dequeue (in the
    # mutex order) is preceded by >= k enqueues: no dequeue finds the queue empty.
    secs, c, nt = oracle.mutex_run(0, T=64, K=200, nthreads=4)
    assert c.tolist() == [64 * 200, 0, 64 * 200, 0]
    assert secs >= 0


def test_mutex_mixed_counts():
    T, K = 256, 100
    bits = synth.mixed_schedule_bits(0, T, K)
    is_enq = synth.schedule_is_enq(bits, T, K)
    secs, c, nt = oracle.mutex_run(1, T, K, sched=bits, nthreads=1)
    # single host thread: logical threads run one after another, so the run is
    # the sequential replay of the thread-major op list
    kinds = is_enq.reshape(-1).astype(np.uint8)
    s, o, final = oracle.seqfifo_run(0, kinds, np.zeros(T * K, np.uint64))
    assert c[0] == int(is_enq.sum()) and c[1] == 0
    assert c[2] == int(((kinds == 0) & (s == 0)).sum())
    assert c[3] == int((s == 2).sum())
    # many host threads: totals of the op kinds are fixed
    secs, c4, nt = oracle.mutex_run(1, T, K, sched=bits, nthreads=8)
    assert c4[0] == c[0] and c4[2] + c4[3] == T * K - c[0]


def test_mutex_split_bounded():
    T = 64
    ops = synth.split_ops_per_thread(10000, T)
    assert ops.sum() == 10000 and ops.max() - ops.min() <= 1
    secs, c, nt = oracle.mutex_run(2, T, 0, producers=32, ops_of=ops, cap=16, nthreads=4)
    assert c[0] + c[1] == ops[:32].sum()
    assert c[2] + c[3] == ops[32:].sum()
    assert c[0] - c[2] <= 16 and c[0] >= c[2]
