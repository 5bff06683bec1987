"""Multi-rank logic of bench.py on CPU ranks (gloo, world size 2): the job time
is the slowest rank's, the whole-job throughput counts the units of all ranks,
and the batched workload's instances are split across the ranks by population
bytes, each rank computing the same split on its own."""
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


def _share_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    from paper_1905_04597_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine, recipe, info = bench.batch_share(rank, world)
    # every rank's share, gathered as instance keys (the recipe is deterministic)
    keys = [recipe.index(r) for r in mine]
    got = [None] * world
    dist.all_gather_object(got, keys)
    nbytes = torch.tensor([float(sum(shard.instance_bytes(r) for r in mine))], dtype=torch.float64)
    dist.all_reduce(nbytes)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, got, info, float(nbytes.item())))


@pytest.mark.parametrize("world", [2, 3])
def test_batch_split_by_bytes_over_gloo_ranks(world):
    sys.path.insert(0, ROOT)
    from paper_1905_04597_gb300 import inputs, shard
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_share_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    recipe = inputs.batched_instances(seed=0)
    sizes = [shard.instance_bytes(r) for r in recipe]
    parts = res[0][1]
    assert all(r[1] == parts for r in res)  # every rank saw the same split
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(recipe)))  # disjoint and complete
    loads = [sum(sizes[i] for i in p) for p in parts]
    assert max(loads) - sum(loads) / world < max(sizes)  # the greedy bound
    assert max(loads) * world / sum(loads) < 1.01  # 256 instances balance well
    assert res[0][3] == pytest.approx(sum(sizes))
    for rank, _, info, _ in res:
        assert info["instances"] == len(parts[rank])


def test_partition_by_bytes_small_case():
    sys.path.insert(0, ROOT)
    from paper_1905_04597_gb300 import shard
    assert shard.partition_by_bytes([5, 4, 3, 3, 3], 2) == [[0, 3], [1, 2, 4]]
    assert shard.partition_by_bytes([1, 1, 1], 1) == [[0, 1, 2]]
    assert shard.partition_by_bytes([7], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        shard.partition_by_bytes([1], 0)
    cfg = dict(k=3, nx=512, ny=256)
    assert shard.instance_bytes(cfg) == 81 * 512 * 256 * 4
    assert shard.instance_bytes(dict(cfg, x_level=1, zv_axes=2)) == 3 * 10 * 512 * 256 * 4
