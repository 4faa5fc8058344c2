"""The replica path of bench.py for N > 1 ranks (one independent solve stream per GPU, no
collective on the data path), exercised as world_size-2 gloo ranks on the CPU: each rank
gets its own seed, the step time is the maximum over ranks, and the whole-job rate counts
every rank's solves."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    slowest = bench.max_over_ranks(local_ms, world, "cpu")
    seeds = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(seeds, torch.tensor([bench.replica_seed(rank)]))
    out[rank] = (slowest, [int(s.item()) for s in seeds], bench.aggregate_rate(world, 5, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_distinct_seeds_and_aggregate_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        slowest, seeds, rate = out[r]
        assert slowest == 150.0                       # max over ranks, seen by every rank
        assert len(set(seeds)) == world               # independent replicas
        assert rate == pytest.approx(world * 5 / 0.150)


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.aggregate_rate(1, 4, 2000.0) == pytest.approx(2.0)
