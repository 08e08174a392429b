"""Counting kernels on the GPU (run with -m gpu): the per-operation event
counts of the fast paths (GQ_OC_*), from a separate instantiation of the run
driver.

Pins:
  * one thread, enqueue-then-dequeue pairs: the counts have a closed form --
    G-LFQ / G-WFQ: per pair four tickets, four fetch-and-adds (a batch of one
    lane), two successful CASes (aq install, fq install), two Consume ORs
    (fq, aq), two first loads of a slot, and one Threshold reset over the
    whole run (aq's Threshold starts at -1, the first install sets it to
    3n - 1 and it never moves again); G-WFQ-YMC: per pair two tickets, two
    successful CASes (the value, the dequeue's claim) and one cell load;
  * concurrent runs: every ticket either completes its ring step or is given
    up (tickets - burned = ring steps = 2 per successful operation for the
    rings, 1 for G-WFQ-YMC, while no operation goes slow); WaveFAA issues
    between tickets / 32 and tickets fetch-and-adds; every completed step is
    one successful CAS or one Consume OR; and the counting
    instantiation still passes the run-log checks against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_01693_gb300 as gq
import synth

from gpu_util import DEV, drain, make_queue, u64

pytestmark = pytest.mark.gpu
KINDS = list(gq.READY_KINDS)


def oc_run(q, mode, T, K=0, sched=None, producers=0, total_ops=0, record=False):
    kmax = K if mode != gq.GQ_RUN_SPLIT else -(-total_ops // T)
    counts = torch.zeros(8, dtype=torch.int64, device=DEV)
    oc = torch.zeros(gq.GQ_OC_N, dtype=torch.int64, device=DEV)
    status = torch.full((kmax, T), -128, dtype=torch.int8, device=DEV) if record else None
    val = torch.zeros((kmax, T), dtype=torch.int64, device=DEV) if record else None
    dsched = torch.from_numpy(sched.view(np.int64)).to(DEV) if sched is not None else None
    gq.gq_run(q.handle, mode, T, ops=K, producers=producers, total_ops=total_ops, sched=dsched, counts=counts,
              status=status, val=val, opcount=oc)
    assert q.sync_status() == 0
    out = {"counts": u64(counts), "oc": dict(zip(gq.OC_NAMES, u64(oc).tolist()))}
    if record:
        out["status"] = status.cpu().numpy()
        out["val"] = u64(val)
    return out


def assert_kind_only_events(kind, oc):
    """Events a kind never produces stay at zero (a count landing in the wrong
    slot would show here)."""
    if kind == "ymc":
        assert oc["rmw"] == oc["threshold"] == oc["catchup"] == 0, oc
    else:
        assert oc["marked"] == 0, oc
        if kind == "lfq":
            assert oc["slow"] == 0, oc


@pytest.mark.parametrize("kind", KINDS)
def test_single_thread_pairs_closed_form(kind):
    K = 200                                             # 100 pairs
    q = make_queue(kind, 1 << 10 if kind != "ymc" else 1 << 12, 8, max_threads=64)
    r = oc_run(q, gq.GQ_RUN_PAIRS, 1, K)
    c, oc = r["counts"], r["oc"]
    assert c[gq.GQ_CNT_ENQ_OK] == K // 2 and c[gq.GQ_CNT_DEQ_OK] == K // 2
    if kind == "ymc":
        want = {"tickets": K, "faa": K, "cas": K, "cas_fail": 0, "rmw": 0, "threshold": 0, "catchup": 0,
                "burned": 0, "loads": K // 2, "slow": 0, "spin": 0, "marked": 0}
    else:
        want = {"tickets": 2 * K, "faa": 2 * K, "cas": K, "cas_fail": 0, "rmw": K, "threshold": 1,
                "catchup": 0, "burned": 0, "loads": K, "slow": 0, "spin": 0, "marked": 0}
    assert oc == want


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("T", [1 << 12, 1 << 16])
def test_concurrent_identities_and_parity(kind, T):
    K = 64
    sched = synth.mixed_schedule_bits(11, T, K)
    q = make_queue(kind, (1 << 20) if kind != "ymc" else (1 << 23), 8, max_threads=T)
    r = oc_run(q, gq.GQ_RUN_MIXED, T, K, sched=sched, record=True)
    c, oc = r["counts"], r["oc"]
    succ = int(c[gq.GQ_CNT_ENQ_OK] + c[gq.GQ_CNT_DEQ_OK])
    steps = succ if kind == "ymc" else 2 * succ
    assert oc["tickets"] // 32 <= oc["faa"] <= oc["tickets"]
    if oc["slow"] == 0:
        assert oc["tickets"] - oc["burned"] == steps
    # a slow-path request completes its operation without a counted CAS
    assert oc["cas"] - oc["cas_fail"] + oc["rmw"] + oc["slow"] >= steps
    assert_kind_only_events(kind, oc)
    kinds = synth.schedule_is_enq(sched, T, K).T.astype(np.uint8).copy()
    rep = oracle.check_log(kinds, r["status"], r["val"], drain(q, 1 << 20))
    assert rep["violations"] == 0, rep


@pytest.mark.parametrize("kind", KINDS)
def test_split_counts_full_and_empty(kind):
    """A 90 % consumer split on a small ring: EMPTY dequeues burn their tickets
    and G-LFQ / G-WFQ catch Tail up; the instantiation stays a correct queue."""
    T, total = 1 << 14, 1 << 19
    q = make_queue(kind, (1 << 10) if kind != "ymc" else (1 << 22), 8, max_threads=T)
    r = oc_run(q, gq.GQ_RUN_SPLIT, T, producers=T // 10, total_ops=total, record=True)
    c, oc = r["counts"], r["oc"]
    assert c[gq.GQ_CNT_DEQ_EMPTY] > 0
    assert oc["burned"] > 0                              # EMPTY tickets (a Threshold < 0 EMPTY takes none)
    assert_kind_only_events(kind, oc)
    from gpu_util import op_kinds
    kinds = op_kinds(gq.GQ_RUN_SPLIT, T, 0, None, T // 10, total)
    rep = oracle.check_log(kinds, r["status"], r["val"], drain(q, 1 << 22))
    assert rep["violations"] == 0, rep


def test_multi_queue_counting_kernel():
    Q, TPQ, OPQ, PPQ = 64, 256, 4000, 128
    caps = np.full(Q, 1 << 10)
    mq = gq.MultiQueue("lfq", caps, 8, TPQ)
    counts = torch.zeros(8, dtype=torch.int64, device=DEV)
    oc = torch.zeros(gq.GQ_OC_N, dtype=torch.int64, device=DEV)
    mq.run(TPQ, PPQ, OPQ, counts, opcount=oc)
    torch.cuda.synchronize()
    c = u64(counts)
    o = dict(zip(gq.OC_NAMES, u64(oc).tolist()))
    succ = int(c[0] + c[2])
    assert o["tickets"] - o["burned"] == 2 * succ
    assert o["tickets"] // 32 <= o["faa"] <= o["tickets"]
    mq.close()
