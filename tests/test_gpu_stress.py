"""Seeded stress of the three queues (run with -m gpu).

A sample of small runs across thread counts, capacities (a ring 2^8 slots
long shared by thousands of threads included), workloads, slow-path settings
and delay injection; every run goes through the oracle's run-log checks and
its ticket checks.
"""
import pytest

import oracle
import paper_2606_01693_gb300 as gq
import synth

from gpu_util import drain, make_queue, run_log

pytestmark = pytest.mark.gpu


def _configs():
    out = []
    for seed in range(700, 708):
        for kind in ("lfq", "wfq", "ymc"):
            T = (1 << 12, 1 << 14)[seed % 2]
            cap = (1 << 8, 1 << 12, 1 << 20)[seed % 3]
            mode = ("mixed", "split")[(seed // 2) % 2]
            opt = {}
            if seed % 4 == 3:
                opt = dict(patience_enq=1, patience_deq=1, help_delay=2) if kind == "wfq" else \
                      dict(patience_enq=0, patience_deq=0) if kind == "ymc" else {}
            out.append((seed, kind, T, cap, mode, opt))
    return out


@pytest.mark.parametrize("seed,kind,T,cap,mode,opt", _configs())
def test_seeded_stress(seed, kind, T, cap, mode, opt):
    q = make_queue(kind, (1 << 26) if kind == "ymc" else cap, 8, max_threads=T, **opt)
    if mode == "mixed":
        K = 32
        r = run_log(q, gq.GQ_RUN_MIXED, T, K, sched=synth.mixed_schedule_bits(seed, T, K), timestamps=True,
                    tickets=True, delay_ns=100 if seed % 3 == 0 else 0)
    else:
        P = (T // 10, T // 2, 9 * T // 10)[seed % 3]
        r = run_log(q, gq.GQ_RUN_SPLIT, T, producers=P, total_ops=24 * T, timestamps=True, tickets=True)
    left = drain(q, 1 << 22)
    rep = oracle.check_log(r["kind"], r["status"], r["val"], left)
    assert rep["violations"] == 0, str(rep)
    tr = oracle.check_tickets(r["kind"], r["status"], r["val"], r["ticket"], r["call"], r["end"],
                              bits=43 if kind == "wfq" else 64)
    assert tr["violations"] == 0, str(tr)
    assert r["counts"][gq.GQ_CNT_ERRORS] == 0
    q.close()
