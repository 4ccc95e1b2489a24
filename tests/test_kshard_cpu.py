"""Coefficients sharded by lattice rows, at world size 2 on the CPU (gloo).

Each rank takes the rows row_partition gives it, computes the coefficients of
those rows with the FP64 oracle (the rows of C are independent: each is a sum
over its own pair set), and one all-gather of the rows (shard.gather_rows,
the path's only exchange step) gives every rank the whole C, which must equal
the unsharded oracle coefficients exactly.  The partition is checked for
disjoint, complete, non-empty ranges and for its balance of pair counts.
"""
import os
import socket

import numpy as np
import pytest

from paper_2310_03979_gb300 import shard

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_C(nk, nw, seeds, mixed):
    import oracle
    from paper_2310_03979_gb300 import workloads as W
    c = W.small_case(nk=nk, nw=nw)
    S = oracle.kaimal_lorentzian(nk, nw, c.kappa_u, c.omega_u, c.U, c.z)
    p = oracle.make_plan(S, c.kappa_u, c.omega_u, eps=0.6, env=oracle.Envelope("gauss", 0.4),
                         beta=0.3, mixed=mixed)
    return np.stack([p.coeffs(s) for s in seeds])  # [n][2][nk][nw] complex


def _worker(rank, world, port, nk, nw, seeds, mixed, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ranges = shard.row_partition(nk, nw, world, mixed)
        full = _oracle_C(nk, nw, seeds, mixed)
        lo, hi = ranges[rank]
        mine = np.zeros_like(full)
        mine[:, :, lo:hi] = full[:, :, lo:hi]  # this rank's rows only
        C = torch.from_numpy(np.stack([mine.real, mine.imag], -1))
        got = shard.gather_rows(C, ranges, rank, dist).numpy()
        out.put((rank, ranges, bool(np.array_equal(got[..., 0] + 1j * got[..., 1], full))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mixed", [False, True])
def test_two_ranks_gather_rows_equals_unsharded(oracle_lib, mixed):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port, world, nk, nw, seeds = _free_port(), 2, 9, 11, (3, 4)
    procs = [ctx.Process(target=_worker, args=(r, world, port, nk, nw, seeds, mixed, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ranges, equal in res:
        assert ranges == shard.row_partition(nk, nw, world, mixed)
        assert equal, f"rank {rank}: gathered coefficients differ from the unsharded ones"


@pytest.mark.parametrize("nk,nw,world,mixed", [
    (256, 512, 2, False), (256, 512, 8, False), (512, 1024, 4, True), (9, 11, 2, False),
    (5, 3, 5, False), (100, 7, 3, True)])
def test_row_partition_disjoint_complete_balanced(nk, nw, world, mixed):
    ranges = shard.row_partition(nk, nw, world, mixed)
    assert ranges[0][0] == 0 and ranges[-1][1] == nk
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c  # contiguous and disjoint
    assert all(b > a for a, b in ranges)  # non-empty
    w = shard.row_pairs(nk, nw, mixed)
    loads = [int(w[a:b].sum()) for a, b in ranges]
    assert sum(loads) == int(w.sum())
    # within one row's pairs of the equal share (the cut is at a row boundary)
    share = w.sum() / world
    assert max(loads) - share <= w.max() + 1


def test_row_pairs_match_pair_counts():
    from paper_2310_03979_gb300 import workloads as W
    for wl in (W.BRIDGE, W.LARGE, W.TINY):
        assert int(shard.row_pairs(wl.n_kappa, wl.n_omega).sum()) == wl.pairs()
    from dataclasses import replace
    m = replace(W.small_case(nk=13, nw=17), interactions="mixed")
    assert int(shard.row_pairs(13, 17, True).sum()) == m.pairs() + m.diff_pairs()
