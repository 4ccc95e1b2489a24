"""The data-parallel path of the benchmark at world size 2, on the CPU (gloo):
each rank samples its own disjoint seeds (weak scaling, no data-path
collective), and the step time reported is the slowest rank's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.rank_seeds(rank, n)
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        slowest = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
        out.put((rank, gathered, slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_disjoint_seeds_and_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port, n, world = _free_port(), 5, 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, slowest in res:
        flat = [s for part in gathered for s in part]
        assert len(flat) == len(set(flat)) == world * n  # disjoint, complete
        assert sorted(flat) == list(range(1, world * n + 1))
        assert slowest == 20.0  # the max over ranks, on every rank
