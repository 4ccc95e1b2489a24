#!/usr/bin/env python
"""Benchmark of the SRM3 stochastic-wave sampler on the bridge-span workload.

One step is one pass of the whole hot path over one batch: build the plan
(discretise the Kaimal-Lorentzian spectrum on the 256 x 512 lattice, the
FP64 pure-spectrum recursion with the eps root search, the stored FP32 W
table), then draw 64 samples (Philox phases, the pair sum, the 2-D inverse
FFT to 512 x 1024 fields).  The metric is pair-terms/s (one pair-term = one
W_ij y_i y_j product for one sheet of one sample) with samples/s beside it.

Ranks shard samples (each rank runs its own plan and its own seeds, no
collective on the data path): weak scaling.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl srm3|reference]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3rd-order SRM wave pair-terms/s & samples/s at stated error; p50/p99 latency"

# DRAM bytes (read + write) of one FP32 pair-sum launch on the 256 x 512 table
# workload with 64 samples, from ncu (dram__bytes_read.sum + dram__bytes_write.sum)
# on the 128 x 256 table case with 64 samples (same two sample groups per
# super-tile), reads scaled by the W table size (x 15.41), writes by the
# coefficient count (x 4).  Valid only for the kernel source it was measured
# on (sha256 prefix of csrc/pairsum.cuh); otherwise reported as null.
PAIRSUM_TRAFFIC = {"bytes": 664.46e6 * 15.41 + 31.16e6 * 4, "source_sha256": "4c3a66e484486035"}
FP32_LANES_PER_SM = 128


def n_sm():
    """Streaming multiprocessors of the current CUDA device
    (cudaDevAttrMultiProcessorCount through torch)."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device())
               .multi_processor_count)


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="srm3", choices=["srm3", "reference"])
    ap.add_argument("--config", default="bridge",
                    choices=["bridge", "bridge_rc", "bridge_sep", "bridge_mixed", "large", "tiny",
                             "prof128",
                             "uneven", "serve", "paper_bridge"],
                    help="workload; bridge is the benchmark line, the others are for "
                         "profiling and checks")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="skip timing the plain FP64 GPU form beside the FP32 line")
    ap.add_argument("--requests", type=int, default=10000,
                    help="serve: number of requests")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def rank_seeds(rank, n):
    """Seeds of rank `rank` when every rank samples n fields (weak scaling):
    disjoint consecutive ranges, 1 + rank n + j."""
    return [1 + rank * n + j for j in range(n)]


def max_over_ranks(x, dist, device):
    """The largest value of x over the ranks (the slowest rank's time), one
    all-reduce on `device` ("cuda" under NCCL, "cpu" under gloo)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def _conv_roofline(wl, n, es, launch_ms):
    """Roofline of the separable pair sum (three FFT self-convolution passes
    over a zero-padded Nk x Nw grid per sheet-sample), bound by HBM: per
    sheet-sample y read twice and C written once (n_kappa n_omega complex
    each), and n_kappa padded rows of Nw complex written, read, written and
    read once more between the passes."""
    nk, nw = wl.n_kappa, wl.n_omega
    Nw = 1 << max(1, (2 * nw - 2).bit_length())
    per_ss = 2 * es * (3 * nk * nw + 4 * nk * Nw)
    nbytes = 2 * n * per_ss
    peak = float(_peaks().get("hbm_gbs", 6800.0))
    gbs = nbytes / (launch_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "traffic": None, "algorithmic_bytes_per_launch": nbytes,
            "per_unit": f"{per_ss} B per sheet-sample (y twice, C once, padded rows 4x)",
            "kernel": "k_conv_rows + k_conv_cols + k_conv_out (one sampling chunk)",
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}


def _pairsum_roofline_fp64(terms_per_s, **extra):
    """Roofline of the plain FP64 pair sum (one thread per output): 6 FP64
    lane operations per pair-term (complex product 2 DMUL + 2 DFMA, weighted
    accumulate 2 DFMA) over the FP64 rate 152 SM x 2 lanes x the maximum SM
    clock (GB300's nominal 1.25 TFLOP/s dense FP64)."""
    sm_max = float(_peaks().get("sm_max_mhz", 2070.0))
    nsm = n_sm()
    lane_rate = 2 * nsm * sm_max * 1e6
    ops = 6.0 * terms_per_s
    out = {"bound": "alu", "achieved": ops / 1e12, "peak": lane_rate / 1e12,
           "unit": "T FP64-pipe lane-ops/s", "frac": ops / lane_rate, "traffic": None,
           "per_unit": "6 FP64-pipe lane-ops per pair-term",
           "peak_source": f"derived: {nsm} SM x 2 FP64 lanes x {sm_max:.0f} MHz"}
    out.update(extra)
    return out


def _pairsum_roofline(terms_per_s, traffic=None, separable=False, sep_share=None, **extra):
    """Roofline object of the FP32 pair sum from its kernel-only rate.

    The bound is the FP32 pipe.  A pair-term is 6 FP32-pipe lane operations
    (2 FMUL + 4 FFMA, 10 flop: the weight times one phasor, then the complex
    product accumulated), so the fraction is pair-terms/s x 6 over the pipe's
    lane-operation rate, 152 SM x 128 lanes x the maximum SM clock.  The same
    rate in flops (10 per pair-term against 2 flop per lane-cycle) is given
    beside it: its ceiling is 10/12 because an FMUL fills a lane slot for one
    flop.  In separable form (the Gaussian envelope's weights folded into the
    phasor rows and the per-row-pair and per-output factors) a pair-term is
    the complex product accumulated alone: 4 FFMA, 8 flop."""
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = n_sm()
    lane_rate = FP32_LANES_PER_SM * nsm * sm_max * 1e6  # lane-ops/s
    # sep_share: the fraction of the pair-terms in separable form (a batch
    # of plans in both forms)
    share = (1.0 if separable else 0.0) if sep_share is None else float(sep_share)
    per_ops, per_flop = 6.0 - 2.0 * share, 10.0 - 2.0 * share
    ops = per_ops * terms_per_s
    flops = per_flop * terms_per_s
    if share == 0.0:
        unit_txt = "6 FP32-pipe lane-ops (2 FMUL + 4 FFMA = 10 flop) per pair-term"
    elif share == 1.0:
        unit_txt = "4 FP32-pipe lane-ops (4 FFMA = 8 flop) per pair-term, separable form"
    else:
        unit_txt = (f"{per_ops:.3f} FP32-pipe lane-ops per pair-term: 4 (4 FFMA) for the "
                    f"{100 * share:.1f} % of pair-terms in separable form, 6 (2 FMUL + 4 FFMA) "
                    "for the rest")
    out = {"bound": "alu", "achieved": ops / 1e12, "peak": lane_rate / 1e12,
           "unit": "T FP32-pipe lane-ops/s", "frac": ops / lane_rate, "traffic": traffic,
           "per_unit": unit_txt,
           "flops": {"achieved": flops / 1e12, "peak": 2.0 * lane_rate / 1e12,
                     "unit": "TFLOP/s", "frac": flops / (2.0 * lane_rate)},
           "peak_source": f"derived: {nsm} SM x {FP32_LANES_PER_SM} FP32 lanes x "
                          f"{sm_max:.0f} MHz (max SM clock of MEASURED_PEAKS.json)"}
    out.update(extra)
    return out


# --------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# oracle on the host cores (CPU baseline / reference arm)

def oracle_baseline(wl, rows=48, seed=1, passes=None):
    """Time the FP64 oracle on a bounded sample of the workload and scale it
    to one full step.  The sample is the first ``rows`` lattice rows (kk <
    rows, all omega): one recursion pass (single-threaded, lexicographic),
    one sample's coefficients (OpenMP over k) and the direct DFT of those rows.
    Recursion and coefficient time scale with the pair count, the DFT with
    the row count; the step is (eps-search passes) recursions plus
    n_samples coefficient sets and DFTs."""
    import numpy as np
    import oracle
    oracle.build()
    dk = wl.kappa_u / wl.n_kappa
    sub = rows
    S = oracle.kaimal_lorentzian(sub, wl.n_omega, sub * dk, wl.omega_u, wl.U, wl.z, wl.z0,
                                 wl.k_vk, wl.lam)
    if wl.envelope != "gauss":  # the workload's tables on the sampled rows
        ta, tb = wl.envelope_tables()
        env = oracle.Envelope("separable", table=np.ascontiguousarray(ta[:sub]),
                              table_b=None if tb is None else np.ascontiguousarray(tb[:sub]))
    else:
        env = oracle.Envelope("gauss", wl.sigma_g * wl.n_kappa / sub)  # same width per index
    eps = 1e-3
    mixed = wl.interactions == "mixed"
    t0 = time.perf_counter()
    if mixed:  # one Gauss-Seidel sweep of the fixed point (it takes about a dozen)
        Sp, _, _ = oracle.recursion_mixed(S, sub * dk, wl.omega_u, eps, env, tol=1.0,
                                          max_sweeps=2)
        t_rec = (time.perf_counter() - t0) / 2
    else:
        Sp, _ = oracle.recursion(S, sub * dk, wl.omega_u, eps, env)
        t_rec = time.perf_counter() - t0
    t0 = time.perf_counter()
    C = oracle.coeffs(S, Sp, sub * dk, wl.omega_u, eps, seed, env, mixed=mixed)
    t_coef = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.field_dft(C, wl.n_x, wl.n_t)
    t_dft = time.perf_counter() - t0
    from paper_2310_03979_gb300.workloads import Workload
    subw = Workload("sub", sub, wl.n_omega, 1.0, 1.0, 1.0, 2.0, 2, 2, (),
                    interactions=wl.interactions)
    sub_pairs = subw.pairs() + subw.diff_pairs()
    full_pairs = wl.pairs() + wl.diff_pairs()
    if passes is None:
        passes = 48  # plain bisection to 1e-13 from the [0, 2^m] bracket
    n = wl.n_samples
    t_step = (passes * full_pairs * (t_rec / sub_pairs)
              + n * full_pairs * (t_coef / sub_pairs)
              + n * (wl.n_kappa / sub) * t_dft)
    terms = 2 * full_pairs * n
    return {
        "value": terms / t_step, "unit": "pair-terms/s", "cores": oracle.num_threads(),
        "kind": "oracle", "step_s": t_step, "samples_per_s": n / t_step,
        "sample": (f"first {sub} of {wl.n_kappa} lattice rows, all {wl.n_omega} omega: one "
                   f"FP64 recursion pass ({t_rec:.2f} s, 1 thread), one sample's coefficients "
                   f"({t_coef:.2f} s) and DFT ({t_dft:.2f} s); scaled by pair count to "
                   f"{passes} eps-search passes + {n} samples of the full lattice"),
    }


# --------------------------------------------------------------------------

def run_uneven(args):
    """The uneven batch: 200 spectra (grids 32..256 per axis, 1..32 samples
    each, seed 4), storage chosen by the autotuner once per lattice shape,
    plans built beforehand (their build time is reported beside the line),
    every step one replay of the captured batch graph (phases of all plans,
    one persistent pair-sum launch, transforms)."""
    import torch
    from paper_2310_03979_gb300 import srm3
    from paper_2310_03979_gb300 import workloads as Wl

    wls = Wl.uneven_batch()
    torch.cuda.init()
    t0 = time.perf_counter()
    tuned = {}
    per_shape = {}
    for wl in wls:
        k = (wl.n_kappa, wl.n_omega)
        per_shape[k] = per_shape.get(k, 0) + wl.n_samples
    for wl in wls:  # one autotune per lattice shape, on that shape's first spectrum, with
        key = (wl.n_kappa, wl.n_omega)  # the samples the batch gives the shape (up to 128)
        if key in tuned:
            continue
        with srm3.Plan.create(wl, storage="table") as p:
            r = srm3.autotune(p.handle, max(1, min(per_shape[key], 128)))
            tuned[key] = {"table_ms": r.table_ms, "recompute_ms": r.recompute_ms,
                          "storage": "table" if r.storage == 1 else "recompute",
                          "tile": f"{r.tile_width} wide"}
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    plans = [srm3.Plan.create(wl, storage="tuned") for wl in wls]
    t_plans = time.perf_counter() - t0
    counts = [wl.n_samples for wl in wls]
    outs = [torch.empty((n, wl.n_x, wl.n_t), dtype=torch.float32, device="cuda")
            for wl, n in zip(wls, counts)]
    seeds = [s for wl in wls for s in wl.seeds]
    stream = torch.cuda.Stream()
    b = srm3.Batch(plans, counts, outs, stream=stream.cuda_stream)
    b.enable_timing(True)
    b.capture()
    for _ in range(args.warmup):
        b.run(seeds)
    b.sync()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    time.sleep(0.3)
    ps = []
    w0 = time.perf_counter()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)  # CUDA events on the batch stream around K back-to-back steps
    for _ in range(args.steps):
        b.run(seeds)
    ev[1].record(stream)
    b.sync()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    wall = time.perf_counter() - w0
    for _ in range(2):  # the pair-sum launch alone (events recorded inside the graph)
        b.run(seeds)
        b.sync()
        ps.append(b.pairsum_ms())
    clocks = sampler.stop()
    terms = b.pair_terms
    nsamp = sum(counts)
    # end to end: host seeds in (inside run), every field copied to pinned host memory
    host = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]
    e2e_ms = []
    for _ in range(max(2, args.steps // 2)):
        t1 = time.perf_counter()
        b.run(seeds)
        b.sync()
        for h, o in zip(host, outs):
            h.copy_(o, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
    ps_ms = statistics.median(ps)
    sep_terms = 0  # pair-terms of plans whose pair sum runs in separable form
    for p, c in zip(plans, counts):
        inf = p.info()
        if inf.recursion_flags & srm3.SRM3_PAIRSUM_SEPARABLE:
            sep_terms += 2 * inf.pairs * c
    choice = {}
    for k, v in tuned.items():
        c = f'{v["storage"]}, {v["tile"]}'
        choice[c] = choice.get(c, 0) + 1
    line = {
        "metric": METRIC, "value": terms / (ms * 1e-3), "unit": "pair-terms/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "uneven_batch_200_spectra_seed4", "spectra": len(wls),
                   "samples_per_step": nsamp, "pair_terms_per_step": terms,
                   "grids": "32..256 per axis (powers of two)",
                   "l2": "inputs smaller than L2 for some spectra; steps are back to back",
                   "step": "one replay of the captured batch graph (phases, one persistent "
                           "pair-sum launch over all spectra, transforms); plans prebuilt"},
        "samples_per_s": nsamp / (ms * 1e-3),
        "wall_ms_per_step": wall * 1e3 / args.steps,
        "plan_build_s_all_spectra": t_plans, "autotune_s": t_tune,
        "autotune_choices": choice,
        "roofline": _pairsum_roofline(terms / (ps_ms * 1e-3), sep_share=sep_terms / terms,
                                      kernel="k_pairsum_f32p (batched, one launch)"),
        "gpu_launches": (3 * len(wls) + 1) * args.steps,
        "clocks": clocks,
        "e2e": {"value": terms / (statistics.median(e2e_ms) * 1e-3), "unit": "pair-terms/s",
                "h2d_bytes_per_step": 8 * nsamp,
                "d2h_bytes_per_step": int(sum(o.numel() * 4 for o in outs)),
                "ms_per_step": statistics.median(e2e_ms)},
    }
    print(json.dumps(line))
    b.destroy()
    for p in plans:
        p.destroy()
    return 0


def run_serve(args):
    """The serving loop: Poisson arrivals (seed 5) of one-sample requests, 90 %
    on the 32 x 32 lattice (64 x 64 field) and 10 % on the 512 x 1024 lattice
    (1024 x 2048 field, W recomputed), spectra from a pool of 32 (U, z) draws
    in the uneven batch's ranges; plan cache under a 150 GB budget; results
    copied to host at completion; FP64 audit of 1 % of the requests."""
    import numpy as np
    import torch
    from paper_2310_03979_gb300 import serve, srm3
    from paper_2310_03979_gb300 import workloads as Wl

    rng = np.random.Generator(np.random.PCG64(5))
    pool = [(float(rng.uniform(20.0, 50.0)), float(rng.uniform(10.0, 60.0))) for _ in range(32)]

    def small(U, z):
        return Wl.Workload("serve_small", 32, 32, 0.5, 4 * math.pi, U, z, 64, 64, (1,),
                           precision="fp32", storage="recompute", target=0.5)

    def large(U, z):
        return Wl.Workload("serve_large", 512, 1024, 0.25, 4 * math.pi, U, z, 1024, 2048, (1,),
                           precision="fp32", storage="recompute", target=0.5)

    torch.cuda.init()
    cache = serve.PlanCache(150e9)
    t0 = time.perf_counter()
    for U, z in pool:  # warm cache: every plan of the pool built before the timed run
        cache.build(small(U, z))
        cache.build(large(U, z))
    t_warm = time.perf_counter() - t0
    # capacity of the large class as the server runs it: one full 64-lane group
    # (32 spectra x 1 sample) with the heavy-slot cap of one CTA per SM
    plans = [cache.lookup(large(U, z)) for U, z in pool]
    outs = [torch.empty((1, 1024, 2048), device="cuda") for _ in pool]
    with srm3.Batch(plans, [1] * len(pool), outs) as b:
        b.set_max_ctas(torch.cuda.get_device_properties(0).multi_processor_count)
        b.run(list(range(len(pool))))
        b.sync()
        t1 = time.perf_counter()
        b.run(list(range(len(pool))))
        b.sync()
        t_group = time.perf_counter() - t1
    del outs
    # and of the small class: one batch of two samples of every pool spectrum
    plans_s = [cache.lookup(small(U, z)) for U, z in pool]
    outs_s = [torch.empty((2, 64, 64), device="cuda") for _ in pool]
    with srm3.Batch(plans_s, [2] * len(pool), outs_s) as b:
        seeds_s = list(range(2 * len(pool)))
        b.run(seeds_s)
        b.sync()
        t1 = time.perf_counter()
        b.run(seeds_s)
        b.sync()
        t_small = (time.perf_counter() - t1) / (2 * len(pool))
    del outs_s
    # requests/s at which the GPU would be 70 % busy with the 10 % / 90 % mix,
    # each class at the per-request cost of a full batch
    rate0 = 0.7 / (0.1 * t_group / len(pool) + 0.9 * t_small)

    def stream(n, rate, gen, rid0):
        gaps = gen.exponential(1.0 / rate, size=n)
        arrivals = np.cumsum(gaps) - gaps[0]
        out = []
        for i in range(n):
            U, z = pool[int(gen.integers(0, len(pool)))]
            wl = large(U, z) if gen.uniform() < 0.1 else small(U, z)
            out.append(serve.Request(rid0 + i, wl, (rid0 + 1_000_000 + i,),
                                     arrival=float(arrivals[i])))
        return out

    # a pilot stream (its own seed) at that rate measures how busy the server
    # really keeps the GPU -- requests arriving alone are sampled alone, at
    # more than a full batch's cost each -- and the rate is scaled to 70 %
    pilot = serve.Server(budget_bytes=150e9, light_slots=1, heavy_slots=1, max_samples=512,
                         cache=cache)
    preqs = stream(max(500, args.requests // 10), rate0,
                   np.random.Generator(np.random.PCG64(55)), 10_000_000)
    pwall = pilot.run(preqs)
    pbusy = pilot.busy / pwall
    pilot.close()
    rate = rate0 * min(1.5, max(0.2, 0.7 / max(pbusy, 1e-3)))
    nreq = args.requests
    reqs = stream(nreq, rate, rng, 0)
    srv = serve.Server(budget_bytes=150e9, light_slots=1, heavy_slots=1, max_samples=512,
                       cache=cache)
    host = {}

    orig_poll = srv._poll

    def poll_with_copy(now):  # results to host as they complete (end to end)
        before = len(srv.finished)
        orig_poll(now)
        for r in srv.finished[before:]:
            h = r.out.cpu()
            if r.rid % 100 == 0:
                host[r.rid] = h
            r.out = None
            r.done = time.perf_counter() - t_run0
    srv._poll = poll_with_copy
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    time.sleep(0.3)
    t_run0 = time.perf_counter()
    wall = srv.run(reqs)
    clocks = sampler.stop()
    srv.close()
    lat = [r.latency * 1e3 for r in reqs]
    lat_s = [r.latency * 1e3 for r in reqs if r.wl.n_kappa == 32]
    lat_l = [r.latency * 1e3 for r in reqs if r.wl.n_kappa == 512]
    pairs = {32: None, 512: None}
    for r in reqs:
        k = r.wl.n_kappa
        if pairs[k] is None:
            pairs[k] = r.wl.pairs()
    terms = sum(2 * pairs[r.wl.n_kappa] for r in reqs)
    # audit: the same seeds through an FP64 plan of the same spectrum
    worst, audited = 0.0, 0
    for rid, h in sorted(host.items()):
        r = reqs[rid]
        wl64 = dataclasses.replace(r.wl, precision="fp64")
        with srm3.Plan.create(wl64) as p64:
            u64 = p64.sample(list(r.seeds)).cpu().double()
            sigma = math.sqrt(p64.info().variance)
        worst = max(worst, float((h.double() - u64).abs().max()) / sigma)
        audited += 1
    nplans = len(cache.plans)
    cache.clear()
    line = {
        "metric": METRIC, "value": terms / wall, "unit": "pair-terms/s", "n_gpus": 1,
        "steps": 1, "warmup": 0, "ms_per_step": wall * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serving_loop_poisson_seed5", "requests": nreq,
                   "mix": "90% 32x32 (64x64 field), 10% 512x1024 (1024x2048 field), 1 sample",
                   "spectra_pool": len(pool), "arrival_rate_per_s": rate,
                   "slots": {"light": 1, "heavy": 1, "heavy_cta_cap": srv.heavy_ctas},
                   "hbm_budget_bytes": 150e9,
                   "step": "the whole request stream, results copied to host at completion"},
        "samples_per_s": nreq / wall,
        "latency_ms": {"p50": serve.percentile(lat, 50), "p99": serve.percentile(lat, 99),
                       "p50_small": serve.percentile(lat_s, 50),
                       "p99_small": serve.percentile(lat_s, 99),
                       "p50_large": serve.percentile(lat_l, 50),
                       "p99_large": serve.percentile(lat_l, 99)},
        "busy_fraction": srv.busy / wall, "batches": srv.batches,
        "plan_cache": {"warm_build_s": t_warm, "plans": nplans,
                       "builds": cache.builds, "evictions": cache.evictions},
        "large_group_ms": t_group * 1e3, "small_request_ms": t_small * 1e3,
        "rate_calibration": {"full_batch_rate_per_s": rate0, "pilot_requests": len(preqs),
                             "pilot_busy_fraction": pbusy},
        "audit": {"requests": audited, "max_abs_du_over_sigma": worst, "tolerance": 1e-4},
        "gpu_launches": srv.launches, "clocks": clocks,
        "e2e": {"value": terms / wall, "unit": "pair-terms/s", "h2d_bytes_per_step": 8 * nreq,
                "d2h_bytes_per_step": int(sum(r.wl.n_x * r.wl.n_t * 4 for r in reqs))},
    }
    print(json.dumps(line))
    return 0


def run_paper_bridge(args):
    """The bridge wind-field experiment of Sec. 5/6: plan build, 1000 samples
    in batches of 50 and their ensemble statistics (moments, histogram) on
    the device; the fields never leave HBM.  The 2nd-order (eps = 0)
    experiment on the same seeds and the exact moments are taken once,
    outside the timed region, for the statistics table."""
    import numpy as np
    import torch
    from paper_2310_03979_gb300 import srm3
    from paper_2310_03979_gb300 import workloads as Wl

    wl = Wl.PAPER_BRIDGE
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    n, B, nbins = wl.n_samples, 50, 240
    seeds = list(wl.seeds)
    out = torch.empty((B, wl.n_x, wl.n_t), dtype=torch.float32, device="cuda")
    probe = srm3.Plan.create(wl, stream=sptr)
    var_exact, m3_exact = probe.moments()
    probe.destroy()
    sig = math.sqrt(var_exact)
    st = srm3.Stats(nbins, -6 * sig, 6 * sig, stream=sptr)
    stats_ms = []

    def experiment(eps=None, timed_stats=False):
        st.reset()
        plan = srm3.Plan.create(wl, stream=sptr, eps=eps)
        srm3.enable_timing(plan.handle, True)
        sms = 0.0
        evs = []
        for b0 in range(0, n, B):
            s = seeds[b0:b0 + B]
            srm3.sample(plan.handle, s, len(s), out.data_ptr())
            if timed_stats:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st.add(out[:len(s)])
                e1.record(stream)
                evs.append((e0, e1))
            else:
                st.add(out[:len(s)])
        r = st.read()
        for e0, e1 in evs:
            sms += e0.elapsed_time(e1)
        t = srm3.get_timings(plan.handle)
        info = plan.info()
        plan.destroy()
        return r, t, info, sms

    for _ in range(args.warmup):
        experiment()
    torch.cuda.synchronize()
    gpu_index = 0
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if cvd.split(",")[0].strip().isdigit():
        gpu_index = int(cvd.split(",")[0])
    sampler = ClockSampler(gpu_index)
    time.sleep(0.3)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    ev0.record(stream)
    recs = [experiment() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - w0) / args.steps
    clocks = sampler.stop()
    ms_per_step = ev0.elapsed_time(ev1) / args.steps
    r3, t3, info, _ = recs[-1]
    # stage split and the stats kernel's own time (one more, untimed run)
    _, _, _, s_ms = experiment(timed_stats=True)
    r2 = experiment(eps=0.0)[0]
    pairs = wl.pairs()
    value = 2 * pairs * n / (ms_per_step * 1e-3)
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    stage_ms = {"plan": info.plan_ms, "recursion": t3.recursion_ms, "phases": t3.phases_ms,
                "pairsum_fft_conv": t3.pairsum_ms, "transform": t3.transform_ms,
                "stats": s_ms}
    # algorithmic HBM bytes per sample: transform (C in; the x stage's
    # n_x x n_omega columns out and in; u out), statistics (u in)
    cNw = 1 << max(1, (2 * wl.n_omega - 2).bit_length())
    per = {"transform": 2 * wl.n_kappa * wl.n_omega * 8 + 2 * wl.n_x * wl.n_omega * 8
                        + wl.n_x * wl.n_t * 4,
           "stats": wl.n_x * wl.n_t * 4,
           # as _conv_roofline: per sheet-sample y twice, C once, padded rows 4x
           "pairsum_fft_conv": 2 * 2 * 4 * (3 * wl.n_kappa * wl.n_omega + 4 * wl.n_kappa * cNw)}
    roofs = {}
    for k, b in per.items():
        if stage_ms[k] > 0:
            gbs = b * n / (stage_ms[k] * 1e-3) / 1e9
            roofs[k] = {"achieved_gbs": gbs, "frac": gbs / hbm, "bytes_per_sample": b}
    dom = max(per, key=lambda k: stage_ms[k])
    line = {
        "metric": METRIC, "value": value, "unit": "pair-terms/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "n_kappa": wl.n_kappa, "n_omega": wl.n_omega,
                   "n_x": wl.n_x, "n_t": wl.n_t, "samples_per_step": n, "batch": B,
                   "l2": "inputs larger than L2 (fields 400 MB per batch)",
                   "step": "plan build + 1000 samples + device statistics"},
        "samples_per_s": n / (ms_per_step * 1e-3),
        "wall_ms_per_step": wall * 1e3,
        "stages_ms_last_step": stage_ms,
        "roofline": {"bound": "hbm", "achieved": roofs[dom]["achieved_gbs"], "peak": hbm,
                     "unit": "GB/s", "frac": roofs[dom]["frac"], "traffic": None,
                     "kernel": dom, "per_unit": f"{per[dom]} B per sample",
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"},
        "stage_rooflines": roofs,
        "statistics": {
            "third_order": {k: r3[k] for k in ("mean", "variance", "skewness", "kurtosis")},
            "second_order": {k: r2[k] for k in ("mean", "variance", "skewness", "kurtosis")},
            "exact": {"mean": 0.0, "variance": var_exact,
                      "skewness": m3_exact / var_exact ** 1.5},
            "values": r3["count"], "histogram_bins": nbins, "range_sigma": 6},
        # per step: spectrum 1, envelope tables 3, sum of S 1, recursion
        # passes, sampling tables 4, conv twiddles 1; per batch of 50 (one
        # sampling chunk): phases, three FFT self-convolution passes, two
        # output FFT stages, statistics pass and merge
        "gpu_launches": args.steps * (1 + 3 + 1 + info.root_passes + info.root_passes_fp32
                                      + 4 + 1 + 8 * math.ceil(n / B)),
        "clocks": clocks,
        "eps": info.eps, "max_sum_b2": info.max_sum_b2,
        "e2e": {"value": 2 * pairs * n / wall, "unit": "pair-terms/s",
                "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * (nbins + 6),
                "ms_per_step": wall * 1e3,
                "note": "wall clock of the experiment through the public API; only "
                        "seeds go in and the statistics come out"},
    }
    st.destroy()
    print(json.dumps(line))
    return 0


def main():
    args = _args()
    if args.config == "uneven" and args.impl != "reference":
        return run_uneven(args)
    if args.config == "paper_bridge" and args.impl != "reference":
        return run_paper_bridge(args)
    if args.config == "serve" and args.impl != "reference":
        return run_serve(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_2310_03979_gb300 import workloads as Wl
    wl = Wl.CONFIGS[args.config]

    if args.impl == "reference":
        if rank != 0:
            return 0
        vals = []
        for i in range(args.warmup + args.steps):
            r = oracle_baseline(wl, rows=32)
            if i >= args.warmup:
                vals.append(r)
        v = statistics.median([x["value"] for x in vals])
        r = vals[-1]
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pair-terms/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * statistics.median([x["step_s"] for x in vals]),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl.name, "n_kappa": wl.n_kappa, "n_omega": wl.n_omega,
                           "samples_per_step": wl.n_samples},
                "samples_per_s": statistics.median([x["samples_per_s"] for x in vals]),
                "cpu_baseline": {"value": v, "unit": "pair-terms/s", "cores": r["cores"],
                                 "kind": "oracle", "sample": r["sample"]},
                "e2e": {"value": v, "unit": "pair-terms/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import numpy as np
    import torch
    from paper_2310_03979_gb300 import srm3

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    n = wl.n_samples
    seeds = rank_seeds(rank, n)
    es = 4 if wl.precision == "fp32" else 8
    dt = torch.float32 if es == 4 else torch.float64
    out = torch.empty((n, wl.n_x, wl.n_t), dtype=dt, device="cuda")
    pairs = wl.pairs() + wl.diff_pairs()
    terms_per_step = 2 * pairs * n
    # mixed interactions: the plan (a fixed-point solve per eps evaluation,
    # seconds at this size) is built once beforehand and its build time is
    # reported beside the line; a step is the sampling batch
    prebuilt = None
    if wl.interactions == "mixed":
        t0 = time.perf_counter()
        prebuilt = srm3.Plan.create(wl, stream=sptr)
        prebuilt_ms = (time.perf_counter() - t0) * 1e3

    def one_step(host_out=None):
        plan = prebuilt or srm3.Plan.create(wl, stream=sptr)
        srm3.enable_timing(plan.handle, True)
        if host_out is None:
            srm3.sample(plan.handle, seeds, n, out.data_ptr())
        else:
            srm3.sample_host(plan.handle, seeds, n, host_out.data_ptr())
        t = srm3.get_timings(plan.handle, reset=prebuilt is not None)
        info = plan.info()
        if prebuilt is None:
            plan.destroy()
        return t, info

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        ids = cvd.split(",")
        if local < len(ids) and ids[local].strip().isdigit():
            gpu_index = int(ids[local])
    sampler = ClockSampler(gpu_index)
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    ev0.record(stream)
    recs = []
    for _ in range(args.steps):
        recs.append(one_step())
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, dist, "cuda")
    ms_per_step = ms / args.steps
    value = terms_per_step * world / (ms_per_step * 1e-3)

    # dominant kernel: the pair sum, timed with events on the plan's stream
    ps_ms = sum(r[0].pairsum_ms for r in recs)
    ps_launch = sum(r[0].pairsum_launches for r in recs)
    ps_terms = sum(r[0].pair_terms for r in recs)
    avg_launch_ms = ps_ms / max(ps_launch, 1)
    terms_per_launch = ps_terms / max(ps_launch, 1)
    info = recs[-1][1]
    t_last = recs[-1][0]
    chunks = math.ceil(n / 128)
    # kernels launched per step (matches the ncu launch list): spectrum 1,
    # envelope tables 2 + g^2 1, separable factors 1 (Gaussian envelope in
    # separable form), recursion index lists 2, the sum of S 2, linear pass
    # 2 + its reduction 2, each recursion pass 1, slope and move of the
    # tables 2 (FP32 plans whose tables were moved), sampling tables 4 (+1
    # for the separable pair sum's), W table 1 if stored; per 128-sample
    # chunk: phases, pair sum, two FFT stages
    flags = info.recursion_flags
    sep_gauss = 1 if (flags & srm3.SRM3_REC_SEPARABLE) and wl.envelope == "gauss" else 0
    moved = 2 if flags & srm3.SRM3_REC_TABLES_MOVED else 0
    # tables interpolated from a three-plane FP64 pass (FP64 plans): 1 kernel
    moved += 1 if flags & srm3.SRM3_REC_TABLES_INTERPOLATED else 0
    # the separable pair sum's scaled tables (FP32 Gaussian plans, either storage)
    sep_tables = 1 if sep_gauss and es == 4 and getattr(wl, "interactions", "sum") == "sum" else 0
    # coarse start of the eps search: its own kernels (subsampled spectrum,
    # envelope tables, index lists, reductions, linear pass, passes), and no
    # linear pass (4 kernels) on the plan's lattice
    coarse = info.coarse_launches - (4 if flags & srm3.SRM3_REC_COARSE_START else 0)
    launches_per_step = (1 + 3 + sep_gauss + 2 + 2 + 4 + (info.root_passes + info.root_passes_fp32)
                         + moved + 4 + sep_tables + (1 if info.storage == 1 else 0) + 4 * chunks
                         + coarse)
    if wl.envelope != "gauss":
        # the bracketing pass is an FP32 pass (counted above) instead of the
        # linear pass; conv twiddles 1; per chunk phases, three FFT
        # self-convolution passes, two output FFT stages
        # (+ the coarse search's kernels: its bound is a pass as well)
        launches_per_step = (1 + 3 + 2 + 2 + (info.root_passes + info.root_passes_fp32)
                             + 4 + 1 + 6 * chunks + info.coarse_launches)
    if prebuilt is not None:
        # sampling only: per chunk phases, sum and difference pair sums, two
        # FFT stages
        launches_per_step = 5 * chunks
    traffic = None
    src = os.path.join(ROOT, "paper_2310_03979_gb300", "csrc", "pairsum.cuh")
    if wl.name.startswith("bridge") and info.storage == 1 and es == 4:
        import hashlib
        with open(src, "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] == PAIRSUM_TRAFFIC["source_sha256"]:
                traffic = PAIRSUM_TRAFFIC["bytes"]

    line = {
        "metric": METRIC, "value": value, "unit": "pair-terms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if es == 4 else "f64", "data": "synthetic",
        "config": {"workload": wl.name, "n_kappa": wl.n_kappa, "n_omega": wl.n_omega,
                   "n_x": wl.n_x, "n_t": wl.n_t, "samples_per_step": n * world,
                   "storage": "table" if info.storage == 1 else "recompute",
                   "precision": wl.precision, "l2": "inputs larger than L2 (W table "
                   f"{info.table_bytes / 1e9:.1f} GB, y {n * 2 * 8 * wl.n_kappa * (wl.n_omega + 128) / 1e6:.0f} MB)",
                   "step": ("plan build (spectrum, FP64 recursion + eps search, W table) + "
                            f"{n}-sample batch") if prebuilt is None else
                           (f"{n}-sample batch on a plan built beforehand (mixed interactions: "
                            f"{prebuilt_ms:.0f} ms to build, the FP64 fixed point of Eq. pure "
                            "solved for every eps of the search)"),
                   "interactions": wl.interactions},
        "samples_per_s": n * world / (ms_per_step * 1e-3),
        "wall_ms_per_step": wall * 1e3 / args.steps,
        "stages_ms_last_step": {"plan_total": info.plan_ms, "recursion": t_last.recursion_ms,
                                "recursion_passes": t_last.recursion_passes,
                                "recursion_fp32_ms": t_last.recursion_fp32_ms,
                                "recursion_fp32_passes": t_last.recursion_passes_fp32,
                                "recursion_fp64_ms": t_last.recursion_fp64_ms,
                                "eps_search_coarse_ms": t_last.coarse_ms,
                                "eps_search_coarse_passes": t_last.recursion_passes_coarse,
                                "table": t_last.table_ms, "phases": t_last.phases_ms,
                                "pairsum": t_last.pairsum_ms,
                                "transform": t_last.transform_ms},
        "sampling_only_pair_terms_per_s": terms_per_step / (
            (t_last.phases_ms + t_last.pairsum_ms + t_last.transform_ms) * 1e-3),
        "roofline": (_conv_roofline(wl, n, es, avg_launch_ms) if wl.envelope != "gauss"
                     else _pairsum_roofline_fp64(terms_per_launch / (avg_launch_ms * 1e-3),
                                                 kernel="k_pairsum_f64") if es == 8
                     else _pairsum_roofline(
            terms_per_launch / (avg_launch_ms * 1e-3), traffic,
            separable=bool(info.recursion_flags & srm3.SRM3_PAIRSUM_SEPARABLE),
            algorithmic_bytes_per_launch=info.table_bytes + n * 2 * 8 * (
                wl.n_kappa * (wl.n_omega + 128) + wl.n_kappa * wl.n_omega),
            kernel="k_pairsum_f32p<table>" if info.storage == 1 else
                   "k_pairsum_f32p<recompute, separable>" if (
                       prebuilt is None and info.recursion_flags & srm3.SRM3_PAIRSUM_SEPARABLE) else
                   "k_pairsum_f32p<recompute>" if prebuilt is None else
                   "k_pairsum_f32p<recompute> + k_pairsum_f32d (sum and difference pairs)")),
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "eps": info.eps, "max_sum_b2": info.max_sum_b2,
    }

    if not args.no_e2e:
        host = torch.empty((n, wl.n_x, wl.n_t), dtype=dt).pin_memory()
        one_step(host)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            one_step(host)
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e_s = max_over_ranks(e2e_s, dist, "cuda")
        line["e2e"] = {"value": terms_per_step * world / e2e_s, "unit": "pair-terms/s",
                       "h2d_bytes_per_step": 8 * n,
                       "d2h_bytes_per_step": n * wl.n_x * wl.n_t * es,
                       "ms_per_step": e2e_s * 1e3}

    if rank == 0 and wl.precision == "fp32" and not args.no_fp64_form and prebuilt is None:
        # the plain FP64 GPU form on the same workload and seeds: sampling only
        # (plans built beforehand), against the FP32 form's sampling stages
        fp64_ms, fp32_ms = [], []
        for prec, sink in (("fp64", fp64_ms), ("fp32", fp32_ms)):
            p = srm3.Plan.create(wl, precision=prec,
                                 storage="recompute" if prec == "fp64" else None, stream=sptr)
            o = torch.empty((n, wl.n_x, wl.n_t),
                            dtype=torch.float64 if prec == "fp64" else torch.float32,
                            device="cuda")
            srm3.sample(p.handle, seeds, n, o.data_ptr())
            for _ in range(2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                srm3.sample(p.handle, seeds, n, o.data_ptr())
                e1.record(stream)
                torch.cuda.synchronize()
                sink.append(e0.elapsed_time(e1))
            p.destroy()
            del o
        line["vs_fp64_form"] = {
            "fp64_samples_per_s": n / (min(fp64_ms) * 1e-3),
            "fp32_samples_per_s": n / (min(fp32_ms) * 1e-3),
            "speedup": min(fp64_ms) / min(fp32_ms),
            "note": "sampling only (plans prebuilt), same workload and seeds"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # a mixed step samples on a prebuilt plan: the oracle's step likewise
        cb = oracle_baseline(wl, rows=128, passes=0 if prebuilt is not None else None)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    if prebuilt is not None:
        prebuilt.destroy()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
