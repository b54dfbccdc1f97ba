"""World-size-2 gloo run of the benchmark's multi-rank host logic (replicas, weak scaling):
disjoint per-rank inputs, max-over-ranks timing, whole-job throughput.  CPU only."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = bench.rank_seeds(rank)
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    worst = bench.max_over_ranks(local_ms, torch.device("cpu"), world)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out[rank] = (worst, bench.throughput(10, world, worst / 1000.0), gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_timing_and_disjoint_inputs():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        worst, value, seeds = out[r]
        assert worst == 150.0
        assert abs(value - 2 * 10 / 0.15) < 1e-9
        assert not set(seeds[0]) & set(seeds[1])
