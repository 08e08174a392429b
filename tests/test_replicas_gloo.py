"""The multi-GPU form is replicas only: each rank runs its own queues and the job
reports the slowest rank's time and the summed operations.  Checked here with two
gloo ranks on the CPU (no GPU, no data-path collective)."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, s = bench.replica_totals(10.0 + 5 * rank, 1000 * (rank + 1))
        out[rank] = (t, s)
        # ranks agree on the job's numbers
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_max_time_and_sum_ops():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == (15.0, 3000.0)


def test_single_process_is_identity():
    import bench
    assert bench.replica_totals(7.5, 42) == (7.5, 42.0)
