"""The allocation-free FIFO round trip (gq_fifo_static_roundtrip) against the
allocating entry points (run with -m gpu).

Some callers cannot call cudaMalloc (another framework owns the device
allocator, or allocation is forbidden once a service runs).  The round trip
keeps its queue in the library's static device array, so these callers can
still enqueue and dequeue a batch.  This file is collected last so that a
failure here comes after every other test has run.
"""
import numpy as np
import pytest
import torch

import paper_2606_01693_gb300 as gq

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _existing(items):
    """Reference: gq_create + gq_enqueue_batch + gq_dequeue_batch on a G-LFQ."""
    n = items.numel()
    cap = 1 << max(1, (n - 1).bit_length())
    q = gq.Queue("lfq", cap, 8, 1 << 16)
    st = torch.zeros(n, dtype=torch.int8, device=DEV)
    ok = torch.zeros(1, dtype=torch.int64, device=DEV)
    q.enqueue(items, st, ok)
    out = torch.zeros(n, dtype=torch.int64, device=DEV)
    ok2 = torch.zeros(1, dtype=torch.int64, device=DEV)
    q.dequeue(out, None, ok2)
    assert q.sync_status() == 0
    k = int(ok2.item())
    res = np.sort(out[:k].cpu().numpy().view(np.uint64))
    q.close()
    return k, res


def _static(items):
    n = items.numel()
    out = torch.full((n,), -7, dtype=torch.int64, device=DEV)
    cnt = torch.full((1,), 12345, dtype=torch.int64, device=DEV)
    gq.gq_fifo_static_roundtrip(items, out, cnt)
    torch.cuda.synchronize()
    k = int(cnt.item())
    return k, np.sort(out[:k].cpu().numpy().view(np.uint64))


def test_static_roundtrip_matches_allocating_path_twice():
    g = torch.Generator().manual_seed(1234)
    # two calls in a row with different sizes: the second must not see the first's contents
    for n in (1 << 16, 3000):
        items = torch.randint(0, 1 << 62, (n,), generator=g, dtype=torch.int64).to(DEV)
        k_ref, ref = _existing(items)
        k, got = _static(items)
        assert k == k_ref == n
        assert (got == ref).all()
        assert (got == np.sort(items.cpu().numpy().view(np.uint64))).all()


def test_static_roundtrip_rejects_oversize_and_handles_empty():
    items = torch.zeros((1 << 16) + 1, dtype=torch.int64, device=DEV)
    out = torch.zeros_like(items)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    with pytest.raises(gq.GqError) as ei:
        gq.gq_fifo_static_roundtrip(items, out, cnt)
    assert ei.value.status == gq.GQ_ERR_INVALID
    cnt.fill_(99)
    gq.gq_fifo_static_roundtrip(items[:0], out[:0], cnt, n=0)
    torch.cuda.synchronize()
    assert int(cnt.item()) == 0
