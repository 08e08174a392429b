"""WaveFAA on the GPU (run with -m gpu): Lemma "WaveFAA preserves ticket order".
Threads chosen by a seeded pattern take one ticket each, on one of two counters
(lanes of a warp mixed, so they are grouped by counter address), at batch widths
1 .. 32.  Each counter's tickets must be exactly 0 .. count-1 (distinct, no gap),
and inside every group of `width` lanes, the lanes on the same counter hold
consecutive tickets increasing with the lane index (the sequential ticket order
of a per-thread fetch-and-add in lane order)."""
import numpy as np
import pytest
import torch

import paper_2606_01693_gb300 as gq
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("width", [1, 2, 8, 32])
@pytest.mark.parametrize("p_take,two", [(1.0, False), (0.6, False), (0.5, True), (0.05, True)])
def test_tickets_distinct_dense_and_lane_ordered(width, p_take, two):
    T = 1 << 16
    u = (synth.splitmix64(17 + width, np.arange(T)) >> np.uint64(40)).astype(np.float64) * 2.0**-24
    take = np.where(u < p_take, 1, 0).astype(np.uint8)
    if two:
        which = (synth.splitmix64(99, np.arange(T)) & np.uint64(1)).astype(np.uint8)
        take = np.where(take == 1, 1 + which, 0).astype(np.uint8)
    d_take = torch.from_numpy(take).cuda()
    counters = torch.zeros(2, dtype=torch.int64, device="cuda")
    tickets = torch.zeros(T, dtype=torch.int64, device="cuda")
    gq.gq_wavefaa_probe(d_take, width, counters, tickets)
    tk = tickets.cpu().numpy().view(np.uint64)
    cn = counters.cpu().numpy()
    for c in (1, 2):
        mine = take == c
        assert cn[c - 1] == mine.sum()
        got = np.sort(tk[mine])
        assert (got == np.arange(mine.sum(), dtype=np.uint64)).all()      # distinct, no gap
    assert (tk[take == 0] == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    # inside each aligned group of `width` lanes: same-counter lanes get consecutive, lane-ordered tickets
    for g0 in range(0, T, width):
        for c in (1, 2):
            lanes = np.flatnonzero(take[g0:g0 + width] == c)
            if len(lanes) > 1:
                seq = tk[g0 + lanes]
                assert (np.diff(seq.astype(np.int64)) == 1).all(), (g0, c, seq)
