"""Multi-rank logic of bench.py on CPU ranks (gloo, world size 2): every rank
runs its own copy of the workload, the job time is the slowest rank's, and
the whole-job throughput counts the units of all ranks."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_setup()
    ms = bench.max_over_ranks(10.0 + 5.0 * rank)  # rank 1 is the slow one
    value = bench.job_throughput(1000, w, ms)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, w, r, local, ms, value))


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, r, local, ms, value in res:
        assert (w, r, local) == (2, rank, rank)
        assert ms == 15.0
        assert value == pytest.approx(2 * 1000 / 0.015)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(100, 1, 2.0) == pytest.approx(50000.0)
