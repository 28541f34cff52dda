"""The N > 1 path of the benchmark (replicas, no data-path collective) on CPU with
gloo, world size 2: max-over-ranks timing and the whole-job rate."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank "times" its own replica; the slowest rank defines the job time
    mine = 1.0 + rank * 0.5
    m = bench.max_over_ranks(mine)
    rate = bench.job_rate(64 * 10, world, m)
    # replicas draw different synthetic inputs of the same distribution
    spec, invs, _ = bench.make_workload("c1", rank)
    q.put((rank, m, rate, int(invs[0]["indices"][:8].sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_timing_and_job_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert all(o[1] == 1.5 for o in out)                     # max over ranks
    assert all(abs(o[2] - 2 * 640 / 1.5) < 1e-9 for o in out)  # whole job: all ranks' units / slowest time
    assert out[0][3] != out[1][3]                              # independent replicas


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_rate(100, 1, 2.0) == 50.0
