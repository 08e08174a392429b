"""Helpers for the GPU parity tests: run the CUDA drivers through the C ABI and
bring their logs back in the shape the oracle's checkers take."""
import numpy as np
import torch

import paper_2606_01693_gb300 as gq
import synth

DEV = "cuda"


def u64(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def make_queue(kind, cap, elem=8, max_threads=1 << 20, **opt):
    return gq.Queue(kind, cap, elem, max_threads, **opt)


def run_log(q, mode, T, K=0, sched=None, producers=0, total_ops=0, block=256, record=True,
            timestamps=False, delay_ns=0, tickets=False):
    """Runs one driver launch; returns (kind, status, val, counts[, call, end][, ticket]) as numpy, op-major."""
    kmax = K if mode != gq.GQ_RUN_SPLIT else -(-total_ops // T)
    status = torch.full((kmax, T), -128, dtype=torch.int8, device=DEV) if record else None
    val = torch.zeros((kmax, T), dtype=torch.int64, device=DEV) if record else None
    call = torch.zeros((kmax, T), dtype=torch.int64, device=DEV) if timestamps else None
    end = torch.zeros((kmax, T), dtype=torch.int64, device=DEV) if timestamps else None
    ticket = torch.zeros((kmax, T), dtype=torch.int64, device=DEV) if tickets else None
    counts = torch.zeros(8, dtype=torch.int64, device=DEV)
    dsched = None
    if sched is not None:
        dsched = torch.from_numpy(sched.view(np.int64)).to(DEV)
    gq.gq_run(q.handle, mode, T, block=block, ops=K, producers=producers, total_ops=total_ops,
              sched=dsched, status=status, val=val, call=call, end=end, counts=counts, delay_ns=delay_ns,
              ticket=ticket)
    st = q.sync_status()
    assert st == 0, gq.status_str(st)
    out = {"counts": u64(counts)}
    if record:
        out["status"] = status.cpu().numpy()
        out["val"] = u64(val)
        out["kind"] = op_kinds(mode, T, K, sched, producers, total_ops)
    if timestamps:
        out["call"] = u64(call)
        out["end"] = u64(end)
    if tickets:
        out["ticket"] = u64(ticket)
    return out


def op_kinds(mode, T, K, sched, producers, total_ops):
    if mode == gq.GQ_RUN_PAIRS:
        k = np.zeros((K, T), np.uint8)
        k[0::2, :] = 1
        return k
    if mode == gq.GQ_RUN_MIXED:
        return synth.schedule_is_enq(sched, T, K).T.astype(np.uint8).copy()
    kmax = -(-total_ops // T)
    nops = synth.split_ops_per_thread(total_ops, T)
    k = np.full((kmax, T), 255, np.uint8)
    rows = np.arange(kmax)[:, None]
    valid = rows < nops[None, :]
    role = np.where(np.arange(T) < producers, 1, 0).astype(np.uint8)
    k[valid] = np.broadcast_to(role, (kmax, T))[valid]
    return k


def drain(q, max_items):
    out = torch.zeros(max_items + 1, dtype=torch.int64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    gq.gq_drain(q.handle, out, cnt)
    assert q.sync_status() == 0
    c = int(cnt.item())
    return u64(out)[:c].copy()
