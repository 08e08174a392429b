"""Batched form on the GPU (run with -m gpu): many independent queues in one
persistent launch, also replayed from a captured CUDA graph, against the
oracle's checks.  The recording instantiation of the persistent kernel stores
every operation's status, value and ticket; each queue's log then goes through
the run-log checks (exactly once with the drained remainder, per-producer
order, no overtaking by the remainder) and the ticket checks (a dequeue carries
its item's enqueue ticket, tickets distinct), queue by queue, as the
single-queue workloads do (Section IV).  The timed kernel's own runs are
checked by their counts and the per-producer order of what is left."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_01693_gb300 as gq
import synth
from paper_2606_01693_gb300 import autotune

from gpu_util import DEV, drain

pytestmark = pytest.mark.gpu
KINDS = list(gq.READY_KINDS)


def _caps(kind, Q, seed, ops_per_queue):
    r = synth.splitmix64(seed, np.arange(Q)) >> np.uint64(40)
    lg = 8 + (r.astype(np.float64) * 2.0**-24 * 9).astype(np.int64)      # log-uniform 2^8 .. 2^16
    caps = (1 << lg)
    if kind == "ymc":                                                       # pool: one cell per ticket
        caps = np.full(Q, 3 * ops_per_queue + (1 << 12))
    return caps


def _check(mq, counts, Q, TPQ, PPQ, OPQ):
    """Counts and the order of what is left (timed kernel: no per-operation log)."""
    c = counts.cpu().numpy().view(np.uint64)
    nops = synth.split_ops_per_thread(OPQ, TPQ)
    assert c[0] + c[1] == Q * nops[:PPQ].sum()
    assert c[2] + c[3] == Q * nops[PPQ:].sum()
    assert c[6] == 0
    left_sum = np.uint64(0)
    for i, q in enumerate(mq.queues):
        assert q.sync_status() == 0
        left = drain(q, int(3 * OPQ + (1 << 16)))
        # FIFO: what is left of each producer comes out of a single-thread drain in sequence order
        prod, seq = left >> np.uint64(32), left & np.uint64(0xFFFFFFFF)
        order = np.argsort(prod, kind="stable")
        same = prod[order][1:] == prod[order][:-1]
        assert (seq[order][1:][same] > seq[order][:-1][same]).all(), i
        assert len(np.unique(left)) == len(left)
        assert ((left >> np.uint64(32)) // np.uint64(TPQ) == np.uint64(i)).all()     # no item crossed queues
        with np.errstate(over="ignore"):
            left_sum = left_sum + left.sum(dtype=np.uint64)
    with np.errstate(over="ignore"):
        assert np.uint64(c[4]) == np.uint64(c[5]) + left_sum          # exactly once, aggregate


class Recorder:
    """Per-operation log buffers of the recording kernel (queue-major, op-major within a queue)."""

    def __init__(self, Q, TPQ, PPQ, OPQ):
        self.Q, self.TPQ, self.PPQ, self.OPQ = Q, TPQ, PPQ, OPQ
        self.K = -(-OPQ // TPQ)
        n = Q * self.K * TPQ
        self.status = torch.full((n,), -128, dtype=torch.int8, device=DEV)
        self.val = torch.zeros(n, dtype=torch.int64, device=DEV)
        self.ticket = torch.zeros(n, dtype=torch.int64, device=DEV)
        nops = synth.split_ops_per_thread(OPQ, TPQ)
        kind = np.full((self.K, TPQ), 255, np.uint8)
        valid = np.arange(self.K)[:, None] < nops[None, :]
        role = np.where(np.arange(TPQ) < PPQ, 1, 0).astype(np.uint8)
        kind[valid] = np.broadcast_to(role, (self.K, TPQ))[valid]
        self.kind = kind

    def args(self):
        return {"status": self.status, "val": self.val, "ticket": self.ticket}

    def check(self, mq, counts, kind_name):
        c = counts.cpu().numpy().view(np.uint64)
        st = self.status.cpu().numpy().reshape(self.Q, self.K, self.TPQ)
        va = self.val.cpu().numpy().view(np.uint64).reshape(self.Q, self.K, self.TPQ)
        tk = self.ticket.cpu().numpy().view(np.uint64).reshape(self.Q, self.K, self.TPQ)
        live = self.kind != 255
        tot = np.zeros(4, np.int64)
        for i, q in enumerate(mq.queues):
            assert q.sync_status() == 0
            left = drain(q, int(3 * self.OPQ + (1 << 16)))
            rep = oracle.check_log(self.kind, st[i], va[i], left)
            assert rep["violations"] == 0, (i, rep)
            tr = oracle.check_tickets(self.kind, st[i], va[i], tk[i], bits=43 if kind_name == "wfq" else 64)
            assert tr["violations"] == 0, (i, tr)
            assert set(np.unique(st[i][live]).tolist()) <= {gq.GQ_OK, gq.GQ_FULL, gq.GQ_EMPTY}
            tot += [rep["enq_ok"], rep["enq_full"], rep["deq_ok"], rep["deq_empty"]]
        assert tot.tolist() == [int(c[0]), int(c[1]), int(c[2]), int(c[3])]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("frac", [0.1, 0.5, 0.9])
def test_recorded_multi_queue_elementwise(kind, frac):
    """256 queues, 1024 threads each, the batched workload's shape (fewer operations)."""
    Q, TPQ, OPQ = 256, 1024, 20000
    PPQ = int(frac * TPQ)
    mq = gq.MultiQueue(kind, _caps(kind, Q, 7, OPQ), 8, TPQ)
    rec = Recorder(Q, TPQ, PPQ, OPQ)
    counts = torch.zeros(8, dtype=torch.int64, device=DEV)
    mq.run(TPQ, PPQ, OPQ, counts, **rec.args())
    rec.check(mq, counts, kind)
    mq.close()


@pytest.mark.parametrize("kind", KINDS)
def test_recorded_graph_replay_elementwise(kind):
    Q, TPQ, OPQ, PPQ = 256, 1024, 10000, 512
    mq = gq.MultiQueue(kind, _caps(kind, Q, 9, OPQ), 8, TPQ)
    rec = Recorder(Q, TPQ, PPQ, OPQ)
    counts = torch.zeros(8, dtype=torch.int64, device=DEV)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        mq.reset()
        mq.run(TPQ, PPQ, OPQ, counts, **rec.args())
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        mq.reset()
        counts.zero_()
        mq.run(TPQ, PPQ, OPQ, counts, **rec.args())
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        rec.check(mq, counts, kind)
    mq.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("frac", [0.1, 0.5, 0.9])
def test_persistent_multi_queue(kind, frac):
    Q, TPQ, OPQ = 64, 256, 20000
    PPQ = int(frac * TPQ)
    mq = gq.MultiQueue(kind, _caps(kind, Q, 5, OPQ), 8, TPQ)
    counts = torch.zeros(8, dtype=torch.int64, device=DEV)
    mq.run(TPQ, PPQ, OPQ, counts)
    _check(mq, counts, Q, TPQ, PPQ, OPQ)
    mq.close()


@pytest.mark.parametrize("kind", KINDS)
def test_graph_replay_matches(kind):
    Q, TPQ, OPQ, PPQ = 32, 256, 10000, 128
    mq = gq.MultiQueue(kind, _caps(kind, Q, 9, OPQ), 8, TPQ)
    counts = torch.zeros(8, dtype=torch.int64, device=DEV)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        mq.reset()
        mq.run(TPQ, PPQ, OPQ, counts)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        mq.reset()
        counts.zero_()
        mq.run(TPQ, PPQ, OPQ, counts)
    for _ in range(3):
        g.replay()
        torch.cuda.synchronize()
        _check(mq, counts, Q, TPQ, PPQ, OPQ)
    mq.close()


def test_autotuner_picks_a_valid_setting(tmp_path, monkeypatch):
    monkeypatch.setenv("GQ_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    Q, TPQ, OPQ, PPQ = 16, 256, 5000, 128
    mq = gq.MultiQueue("lfq", _caps("lfq", Q, 3, OPQ), 8, TPQ)
    best = autotune.tune_multi(mq, TPQ, PPQ, OPQ, widths=(32, 8), blocks_per_sm=(0, 2), backoffs=(0, 200), reps=1)
    assert best["batch_width"] in (32, 8) and best["mops"] > 0 and len(best["table"]) == 8
    again = autotune.tune_multi(mq, TPQ, PPQ, OPQ, widths=(32, 8), blocks_per_sm=(0, 2), backoffs=(0, 200), reps=1)
    assert again["cached"] and again["batch_width"] == best["batch_width"]
    counts = torch.zeros(8, dtype=torch.int64, device=DEV)
    mq.reset()
    mq.run(TPQ, PPQ, OPQ, counts, blocks=best["blocks"])
    _check(mq, counts, Q, TPQ, PPQ, OPQ)
    mq.close()


def test_wfq_help_delay_tuning_and_bound(tmp_path, monkeypatch):
    """The G-WFQ help delay D is a tuned knob; a D that would break some queue's
    cycle-tag bound R > D k / n + 6 is refused and skipped by the autotuner, and
    the tuned setting still passes the run checks."""
    monkeypatch.setenv("GQ_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    Q, TPQ, OPQ, PPQ = 8, 256, 4000, 128
    mq = gq.MultiQueue("wfq", _caps("wfq", Q, 5, OPQ), 8, TPQ)
    R = 1 << 19
    too_big = (R - 6) * min(q.capacity for q in mq.queues) // TPQ + 1
    with pytest.raises(gq.GqError) as ei:
        mq.prepare(help_delay=too_big)
    assert ei.value.status == gq.GQ_ERR_TOO_MANY_THREADS
    best = autotune.tune_multi(mq, TPQ, PPQ, OPQ, widths=(32,), blocks_per_sm=(0,), backoffs=(0,), reps=1,
                               patiences=[(16, 64)], help_delays=[0, 1, too_big])
    assert {r["help_delay"] for r in best["table"]} == {0, 1}
    counts = torch.zeros(8, dtype=torch.int64, device=DEV)
    mq.reset()
    mq.run(TPQ, PPQ, OPQ, counts, blocks=best["blocks"])
    _check(mq, counts, Q, TPQ, PPQ, OPQ)
    mq.close()
