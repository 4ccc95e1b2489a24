"""Plans restricted to a range of lattice rows (one shard of a job that splits
the W table and the pair sum by rows across devices), on one GPU.

Each row's coefficients are a sum over its own pair set, computed by the same
work units whether or not the plan holds the other rows, so the shards' rows
stitched together must equal the unsharded coefficients bit for bit, and the
transform of the stitched C the unsharded fields; the shards' W tables add up
to the unsharded table.  The gather between devices is the host-side
shard.gather_rows (tested at world size 2 on gloo in test_kshard_cpu.py).
"""
from dataclasses import replace

import pytest

from paper_2310_03979_gb300 import shard, srm3
from paper_2310_03979_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ("table_fp32", W.small_case(nk=40, nw=70, nx=64, nt=256, seeds=(1, 2, 3)), "table", 3),
    ("recompute_fp32", W.small_case(nk=40, nw=70, nx=64, nt=256, seeds=(1, 2, 3)), "recompute", 2),
    ("fp64", W.small_case(nk=24, nw=37, nx=32, nt=128, seeds=(4, 5), precision="fp64"),
     "recompute", 2),
    ("mixed_fp32", replace(W.small_case(nk=33, nw=20, nx=64, nt=64, seeds=(6, 7)),
                           interactions="mixed", sigma_g=0.4), "recompute", 2),
]


@pytest.mark.parametrize("name,wl,storage,world", CASES, ids=[c[0] for c in CASES])
def test_row_shards_stitch_to_the_unsharded_coefficients(name, wl, storage, world):
    eps = 0.6
    seeds = list(wl.seeds)
    mixed = wl.interactions == "mixed"
    ranges = shard.row_partition(wl.n_kappa, wl.n_omega, world, mixed)
    with srm3.Plan.create(wl, storage=storage, eps=eps) as full:
        ref_C = full.coeffs(seeds)
        ref_u = full.sample(seeds)
        full_info = full.info()
        torch.cuda.synchronize()
        C = torch.full_like(ref_C, float("nan"))
        table_bytes, pairs = 0.0, 0
        for lo, hi in ranges:
            with srm3.Plan.create(wl, storage=storage, eps=eps, rows=(lo, hi)) as p:
                part = p.coeffs(seeds)
                torch.cuda.synchronize()
                C[:, :, lo:hi] = part[:, :, lo:hi]
                info = p.info()
                table_bytes += info.table_bytes
                pairs += info.pairs
                with pytest.raises(srm3.SRM3Error) as ei:  # fields need every shard
                    p.sample(seeds)
                assert ei.value.code == -8
        assert torch.equal(C, ref_C)
        u = full.field_from_coeffs(C)
        torch.cuda.synchronize()
        assert torch.equal(u, ref_u)
    assert table_bytes == full_info.table_bytes
    assert pairs == full_info.pairs


def test_row_range_arguments_are_checked():
    wl = W.small_case(nk=12, nw=12)
    for rows in ((3, 3), (-1, 4), (5, 13), (6, 2)):
        with pytest.raises(srm3.SRM3Error) as ei:
            srm3.Plan.create(wl, eps=0.5, rows=rows)
        assert ei.value.code == -1
    sep = replace(W.BRIDGE_SEP, n_kappa=12, n_omega=12, n_x=16, n_t=32)
    with pytest.raises(srm3.SRM3Error) as ei:
        srm3.Plan.create(sep, eps=0.5, rows=(0, 6))
    assert ei.value.code == -8
