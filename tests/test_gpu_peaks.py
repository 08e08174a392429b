"""Atomic-peak probes on the GPU (run with -m gpu): every pattern runs and reports a
positive rate, and hot counters 4 KB apart add up their rates while counters 128 B
apart share L2 slices (the reason the queue's control lines are 4 KB apart)."""
import pytest
import torch

import paper_2606_01693_gb300 as gq

pytestmark = pytest.mark.gpu


def _rate(pattern, iters=64):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    buf = torch.zeros(1 << 21, dtype=torch.int64, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    blocks, threads = sms * 8, 256
    gq.gq_atomic_peak(pattern, blocks, threads, iters, buf, sink)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    gq.gq_atomic_peak(pattern, blocks, threads, iters, buf, sink)
    e1.record()
    e1.synchronize()
    ops = blocks * threads * iters
    if pattern in (gq.GQ_PEAK_SAME_ADDR_FAA, gq.GQ_PEAK_SPREAD_FAA, gq.GQ_PEAK_PACKED_FAA):
        ops //= 32
        # every fetch-add landed: the counters hold the two launches' increments
        words = {gq.GQ_PEAK_SAME_ADDR_FAA: [0], gq.GQ_PEAK_SPREAD_FAA: [512 * c for c in range(16)],
                 gq.GQ_PEAK_PACKED_FAA: [16 * c for c in range(16)]}[pattern]
        assert int(buf[words].sum()) == 2 * ops
    return ops / (e0.elapsed_time(e1) * 1e-3)


@pytest.mark.parametrize("pattern", range(6))
def test_pattern_runs(pattern):
    assert _rate(pattern) > 0


def test_spread_counters_beat_packed_counters():
    assert _rate(gq.GQ_PEAK_SPREAD_FAA) > 1.5 * _rate(gq.GQ_PEAK_PACKED_FAA)
