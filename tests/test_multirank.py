"""The multi-GPU form of the benchmark is replicas only: each rank solves its
own copy of the workload and the job's value is all ranks' cell-steps over
the slowest rank's time.  The cross-rank step (an all-reduce MAX of the
timings) runs here on world_size-2 gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = [1.25, 2.5][rank]
    t_max = bench.max_over_ranks(t_local, world, "cpu")
    v = bench.job_value(1_000_000, 4, world, t_max)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t_max, v))


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, v in out:
        assert t_max == 2.5                               # the slowest rank's time
        assert v == pytest.approx(1e6 * 4 * 2 / 2.5 / 1e9)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.job_value(10, 3, 1, 2.0) == pytest.approx(15e-9)
