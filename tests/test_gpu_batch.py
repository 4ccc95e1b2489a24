"""Batches of plans (one persistent pair-sum launch over uneven lattices and
sample counts, optionally replayed from a captured CUDA graph) and the
storage autotuner, through the C ABI.

A batch runs the same kernels with the same per-unit arithmetic as
srm3_sample, so its fields must be bit-identical to each plan's own
srm3_sample for the same seeds, whatever the mix."""
import pytest

from paper_2310_03979_gb300 import srm3
from paper_2310_03979_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIX = [  # (lattice, storage, samples); the two 24 x 37 spectra form one shape group
    (W.small_case(nk=24, nw=37, nx=64, nt=128, precision="fp32"), "recompute", 3),
    (W.small_case(nk=24, nw=37, nx=64, nt=128, precision="fp32", U=45.0, target=0.4),
     "recompute", 2),
    (W.small_case(nk=32, nw=16, nx=32, nt=32, precision="fp32", U=25.0, target=0.3), "table", 1),
    (W.small_case(nk=17, nw=40, nx=32, nt=128, precision="fp32", z=45.0, target=0.65),
     "recompute", 5),
    (W.small_case(nk=16, nw=16, nx=16, nt=32, precision="fp64"), "recompute", 2),
    (W.small_case(nk=40, nw=70, nx=64, nt=256, precision="fp32", target=0.1), "table", 32),
]


def _dtype(wl):
    return torch.float32 if wl.precision == "fp32" else torch.float64


def _seed_lists(base):
    seeds = []
    for i, (_, _, n) in enumerate(MIX):
        seeds.append([base + i + 1000 * j + 7 for j in range(n)])
    return seeds


def test_batch_matches_srm3_sample_direct_and_graph():
    plans = [srm3.Plan.create(wl, storage=st) for wl, st, _ in MIX]
    try:
        outs = [torch.full((n, wl.n_x, wl.n_t), float("nan"), dtype=_dtype(wl), device="cuda")
                for wl, _, n in MIX]
        with srm3.Batch(plans, [n for _, _, n in MIX], outs) as b:
            assert b.pair_terms == sum(2 * p.info().pairs * n for p, (_, _, n) in zip(plans, MIX))
            b.enable_timing(True)
            for base, capture in ((1, False), (50, True), (90, False)):
                if capture:
                    b.capture()
                seeds = _seed_lists(base)
                b.run([s for ss in seeds for s in ss])
                b.sync()
                assert b.pairsum_ms() > 0.0
                for p, o, ss in zip(plans, outs, seeds):
                    ref = p.sample(ss)
                    torch.cuda.synchronize()
                    assert torch.equal(o, ref), (p.nk, p.nw, base)
    finally:
        for p in plans:
            p.destroy()


def test_batch_holds_workspace_and_checks_arguments():
    wl = W.small_case(nk=24, nw=37, nx=64, nt=128, precision="fp64")
    with srm3.Plan.create(wl, storage="recompute") as p:  # FP64: outside shape groups
        out = torch.empty((2, wl.n_x, wl.n_t), dtype=torch.float64, device="cuda")
        with pytest.raises(srm3.SRM3Error):
            srm3.Batch([p, p], [1, 1], [out, out])  # one plan, one workspace
        with pytest.raises(srm3.SRM3Error):
            srm3.Batch([p], [0], [out])
        with srm3.Batch([p], [2], [out]) as b:
            b.run([1, 2])
            b.sync()
            with pytest.raises(srm3.SRM3Error):  # the workspace may not grow under the batch
                p.sample(list(range(1, 101)))
        u = p.sample(list(range(1, 101)))  # and may again once the batch is gone
        torch.cuda.synchronize()
        assert torch.isfinite(u).all()


def test_autotune_chooses_a_storage_and_tuned_plans_use_it():
    wl = W.small_case(nk=48, nw=96, nx=64, nt=256, precision="fp32", storage="table")
    seeds = [3, 4, 5, 6]
    with srm3.Plan.create(wl, storage="recompute") as ref_plan:
        ref = ref_plan.sample(seeds)
        torch.cuda.synchronize()
    with srm3.Plan.create(wl, storage="table") as p:
        r = srm3.autotune(p.handle, 4)
        assert r.storage in (srm3.SRM3_STORAGE_TABLE, srm3.SRM3_STORAGE_RECOMPUTE)
        assert r.table_ms > 0 and r.recompute_ms > 0 and r.samples == 4
        assert p.info().storage == r.storage
        assert (p.info().table_bytes > 0) == (r.storage == srm3.SRM3_STORAGE_TABLE)
        u = p.sample(seeds)
        torch.cuda.synchronize()
        scale = ref.abs().max().item()
        assert (u - ref).abs().max().item() <= 2e-5 * scale
    with srm3.Plan.create(wl, storage="tuned") as q:
        assert q.info().storage == r.storage
    fp64 = W.small_case(nk=16, nw=16, nx=16, nt=32, precision="fp64")
    with srm3.Plan.create(fp64) as d:
        with pytest.raises(srm3.SRM3Error):
            srm3.autotune(d.handle, 2)


def test_uneven_batch_spectra_against_oracle(oracle_lib):
    """The uneven-batch workload's own spectra (seed 4, the benchmark's draw):
    its smallest lattices, autotuned storage as in the benchmark, through one
    captured batch graph, against the FP64 oracle (its own bisection on each
    spectrum's target, coefficients and direct DFT), max|du| <= 1e-4 sigma_u."""
    import math

    import numpy as np

    import oracle

    spectra = [wl for wl in W.uneven_batch() if wl.n_kappa * wl.n_omega <= 32 * 64][:4]
    assert len(spectra) >= 3
    plans = [srm3.Plan.create(wl, storage="recompute") for wl in spectra]
    try:
        outs = [torch.full((wl.n_samples, wl.n_x, wl.n_t), float("nan"), device="cuda")
                for wl in spectra]
        with srm3.Batch(plans, [wl.n_samples for wl in spectra], outs) as b:
            b.capture()
            b.run([s for wl in spectra for s in wl.seeds])
            b.sync()
        worst = 0.0
        for wl, o in zip(spectra, outs):
            S = oracle.kaimal_lorentzian(wl.n_kappa, wl.n_omega, wl.kappa_u, wl.omega_u,
                                         wl.U, wl.z, wl.z0, wl.k_vk, wl.lam)
            op = oracle.make_plan(S, wl.kappa_u, wl.omega_u, target=wl.target,
                                  env=oracle.Envelope("gauss", wl.sigma_g))
            sig = math.sqrt(op.moments()[0])
            u = o.cpu().double().numpy()
            for i, s in enumerate(wl.seeds[:3]):
                err = np.abs(u[i] - op.field(s, wl.n_x, wl.n_t)).max() / sig
                worst = max(worst, err)
                assert err <= 1e-4, (wl.name, s, err)
        print(f"uneven-batch spectra {[w.name for w in spectra]}: max|du|/sigma_u = "
              f"{worst:.3e} against the FP64 oracle")
    finally:
        for p in plans:
            p.destroy()


@pytest.mark.parametrize("storage,n", [("table", 3), ("recompute", 3), ("recompute", 40)])
def test_tile_widths_give_identical_fields(storage, n):
    """The 16-wide work unit (two compute warps) walks each output's chunks
    and register blocks as the 32-wide one does: the fields are the same bit
    for bit (full- and half-group modes, stored and recomputed W)."""
    wl = W.small_case(nk=40, nw=70, nx=64, nt=256, precision="fp32")
    seeds = list(range(11, 11 + n))
    with srm3.Plan.create(wl, storage=storage) as p:
        assert p.info().tile_width == 32
        ref = p.sample(seeds)
        p.set_tile_width(16)
        assert p.info().tile_width == 16
        got = p.sample(seeds)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        with pytest.raises(srm3.SRM3Error):
            p.set_tile_width(24)


def test_batch_with_both_tile_widths():
    """A batch whose plans were set to different tiles runs one launch in the
    tile of most of its pair-terms; every plan's fields equal its own
    srm3_sample (in its own tile)."""
    plans = [srm3.Plan.create(wl, storage=st) for wl, st, _ in MIX]
    try:
        for i, p in enumerate(plans):
            if p.precision == "fp32" and i % 2 == 1:
                p.set_tile_width(16)
        outs = [torch.full((n, wl.n_x, wl.n_t), float("nan"), dtype=_dtype(wl), device="cuda")
                for wl, _, n in MIX]
        with srm3.Batch(plans, [n for _, _, n in MIX], outs) as b:
            seeds = _seed_lists(300)
            b.capture()
            b.run([s for ss in seeds for s in ss])
            b.sync()
            for p, o, ss in zip(plans, outs, seeds):
                ref = p.sample(ss)
                torch.cuda.synchronize()
                assert torch.equal(o, ref), (p.nk, p.nw)
    finally:
        for p in plans:
            p.destroy()


def test_autotune_times_every_storage_and_tile():
    wl = W.small_case(nk=32, nw=64, nx=64, nt=128, precision="fp32", storage="table")
    with srm3.Plan.create(wl, storage="table") as p:
        r = srm3.autotune(p.handle, 8)
        assert r.tile_width in (16, 32)
        for t in (r.table_ms_w32, r.table_ms_w16, r.recompute_ms_w32, r.recompute_ms_w16):
            assert t > 0
        assert r.recompute_ms == min(r.recompute_ms_w32, r.recompute_ms_w16)
        assert p.info().tile_width == r.tile_width
    with srm3.Plan.create(wl, storage="recompute") as q:  # later plans of the shape take the tile
        assert q.info().tile_width == r.tile_width


def test_stored_table_plans_of_one_shape_share_lanes():
    """Plans with stored W tables of one lattice shape form a shape group (the
    table holds the pair envelopes of the shape; each sample applies its own
    spectrum's pair factor): the batch equals each plan sampled alone."""
    wls = [W.small_case(nk=24, nw=37, nx=64, nt=128, U=U, target=t)
           for U, t in ((30.0, 0.5), (44.0, 0.35), (22.0, 0.6))]
    counts = [3, 1, 2]
    plans = [srm3.Plan.create(wl, storage="table") for wl in wls]
    try:
        assert all(p.info().table_bytes > 0 for p in plans)
        outs = [torch.full((n, 64, 128), float("nan"), device="cuda") for n in counts]
        seeds = [[5 + 10 * i + j for j in range(n)] for i, n in enumerate(counts)]
        with srm3.Batch(plans, counts, outs) as b:
            b.run([s for ss in seeds for s in ss])
            b.sync()
            # one shape group: the batch's own buffers hold its samples
            assert b.device_bytes >= 24 * (37 + 128) * 64 * 8
        for p, o, ss in zip(plans, outs, seeds):
            ref = p.sample(ss)
            torch.cuda.synchronize()
            assert torch.equal(o, ref)
    finally:
        for p in plans:
            p.destroy()
