"""Parity at the benchmark sizes.

* Bridge workload (256 x 512, the launch configuration of bench.py: FP32
  plan, stored W table, 64 samples): eps, q and sum b^2 at 64 lattice points,
  the exact variance, and the coefficients of seeds 1..4 at those points,
  against the FP64 oracle's values in tests/golden/bridge_256x512.json
  (written by tests/golden/make_bridge_golden.py, which calls only oracle/).
  Tolerances: eps 2e-8 relative and tables 1e-7 relative (an FP32 plan meets
  the target to 1e-9); coefficients 2e-6 of max|C| (FP32 accumulation).
* The FP32 fields against the GPU's plain FP64 form on all 64 samples:
  max|du| <= 1e-4 sigma_u.
* Large grid (512 x 1024, W recomputed, 16 samples): FP32 against FP64,
  max|du| <= 1e-4 sigma_u, and the ensemble skewness of the two within 1e-4.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2310_03979_gb300 import srm3
from paper_2310_03979_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bridge_256x512.json")


def _golden():
    if not os.path.exists(GOLDEN):
        pytest.skip("tests/golden/bridge_256x512.json not written yet")
    with open(GOLDEN) as f:
        return json.load(f)


def test_bridge_plan_against_oracle():
    g = _golden()
    with srm3.Plan.create(W.BRIDGE) as p:
        info = p.info()
        S, q, sb2 = p.tables()
    assert abs(info.eps - g["eps"]) <= 2e-8 * g["eps"]
    assert abs(info.max_sum_b2 - g["max_sum_b2"]) <= 1e-9
    # the eps search started from the root on the 64 x 64 lattice of every
    # fourth kappa and eighth omega point, bracketed by one FP32 pass here
    # (four planes over the window around that root) and finished by one FP64
    # pass with the tables moved to the root
    assert info.recursion_flags & srm3.SRM3_REC_COARSE_START
    assert (info.coarse_fk, info.coarse_fw) == (4, 8)
    assert (info.root_passes_fp32, info.root_passes) == (1, 1)
    assert abs(info.variance - g["variance"]) <= 1e-12 * g["variance"]
    pts = [tuple(x) for x in g["points"]]
    qg, sg = np.array(g["q"]), np.array(g["sum_b2"])
    qq = np.array([q[a, b] for a, b in pts])
    ss = np.array([sb2[a, b] for a, b in pts])
    np.testing.assert_allclose(qq, qg, rtol=1e-7)
    np.testing.assert_allclose(ss, sg, rtol=1e-7, atol=1e-12)


def test_bridge_coefficients_seeds_1_to_4_against_oracle():
    g = _golden()
    pts = [tuple(x) for x in g["points"]]
    with srm3.Plan.create(W.BRIDGE) as p:
        C = p.coeffs([1, 2, 3, 4]).cpu().numpy()
    C = C[..., 0] + 1j * C[..., 1]
    for i, s in enumerate((1, 2, 3, 4)):
        ref = np.array(g["coeffs"][str(s)])  # [sheet][point][re, im]
        ref = ref[..., 0] + 1j * ref[..., 1]
        got = np.array([[C[i, sh, a, b] for a, b in pts] for sh in range(2)])
        scale = g["coeffs_max_abs_" + str(s)]
        assert np.abs(got - ref).max() <= 2e-6 * scale, s


def _fields(wl, precision, seeds):
    with srm3.Plan.create(wl, precision=precision,
                          storage=wl.storage if precision == "fp32" else "recompute") as p:
        u = p.sample(seeds)
        torch.cuda.synchronize()
        return u.double(), math.sqrt(p.info().variance)


def test_bridge_fp32_against_fp64_all_64_samples():
    seeds = list(W.BRIDGE.seeds)
    u32, sig = _fields(W.BRIDGE, "fp32", seeds)
    u64, _ = _fields(W.BRIDGE, "fp64", seeds)
    err = (u32 - u64).abs().max().item() / sig
    print(f"bridge, 64 samples: max|du|/sigma_u = {err:.3e}")
    assert err <= 1e-4


def _skew(u):
    m = u.mean()
    d = u - m
    return ((d ** 3).mean() / (d ** 2).mean() ** 1.5).item()


def test_large_fp32_against_fp64_16_samples():
    seeds = list(W.LARGE.seeds)
    u32, sig = _fields(W.LARGE, "fp32", seeds)
    u64, _ = _fields(W.LARGE, "fp64", seeds)
    err = (u32 - u64).abs().max().item() / sig
    s32, s64 = _skew(u32), _skew(u64)
    print(f"large, 16 samples: max|du|/sigma_u = {err:.3e}, skewness {s32:.6f} vs {s64:.6f}")
    assert err <= 1e-4
    assert abs(s32 - s64) <= 1e-4
