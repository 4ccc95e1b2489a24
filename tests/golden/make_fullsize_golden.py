"""Writes tests/golden/fields_fullsize.json: oracle field values and
coefficients at the benchmark sizes, computed by the FP64 oracle alone.

  * bridge (256 x 512 lattice, 512 x 1024 fields): the oracle's own eps from
    tests/golden/bridge_256x512.json (its bisection to 1e-13 on max sum b^2,
    written by make_bridge_golden.py), one oracle recursion pass at that eps,
    the full-lattice coefficients of seeds 1..4 and, from them, the field
    u(mx dx, mt dt) at 256 seeded output points by the plain double sum over
    all coefficients (FFT form, Sec. 4.3; no FFT anywhere).
  * large (512 x 1024 lattice, 1024 x 2048 fields): a stated fixed scale
    eps = 1.6 (no search, no GPU value), one oracle recursion pass, q and
    sum b^2 at 64 lattice points, the coefficients of seed 1 at those points
    and the field of seed 1 at 256 output points, as above.

Nothing here comes from the CUDA path.  Takes about half an hour on 8 cores
(the recursion is sequential in lexicographic order: about 45 s per pass on
the bridge lattice, 12 min on the large one).

    python tests/golden/make_fullsize_golden.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2310_03979_gb300 import workloads as W  # noqa: E402

LARGE_EPS = 1.6
SEEDS_BRIDGE = (1, 2, 3, 4)


def lattice_points(nk, nw, n_random=56, seed=20231003):
    """Corners, edges and a seeded random spread of lattice points."""
    pts = {(0, 1), (1, 0), (1, 1), (nk - 1, nw - 1), (nk - 1, 1), (1, nw - 1),
           (nk // 2, nw // 2), (nk - 1, nw // 2)}
    rng = np.random.default_rng(seed)
    while len(pts) < 8 + n_random:
        pts.add((int(rng.integers(0, nk)), int(rng.integers(1, nw))))
    return sorted(pts)


def output_points(nx, nt, n_random=248, seed=19):
    """Corners, the centre and a seeded random spread of (mx, mt) points."""
    pts = {(0, 0), (0, nt - 1), (nx - 1, 0), (nx - 1, nt - 1), (nx // 2, nt // 2),
           (1, 1), (nx // 2 - 1, nt - 1), (nx - 1, nt // 2 + 1)}
    rng = np.random.default_rng(seed)
    while len(pts) < 8 + n_random:
        pts.add((int(rng.integers(0, nx)), int(rng.integers(0, nt))))
    return sorted(pts)


def spectrum(wl):
    return oracle.kaimal_lorentzian(wl.n_kappa, wl.n_omega, wl.kappa_u, wl.omega_u, wl.U,
                                    wl.z, wl.z0, wl.k_vk, wl.lam)


def main():
    oracle.build()
    t0 = time.time()
    with open(os.path.join(HERE, "bridge_256x512.json")) as f:
        bridge_eps = json.load(f)["eps"]
    out = {"source": "oracle/ (lexicographic recursion at a given eps, coefficients, "
                     "field by the plain double sum at selected points)",
           "threads": oracle.num_threads()}

    # bridge: fields of seeds 1..4 at output points
    wl = W.BRIDGE
    env = oracle.Envelope("gauss", wl.sigma_g)
    op = oracle.make_plan(spectrum(wl), wl.kappa_u, wl.omega_u, eps=bridge_eps, env=env,
                          beta=wl.beta)
    var, _ = op.moments()
    opts = output_points(wl.n_x, wl.n_t)
    mx = np.array([p[0] for p in opts])
    mt = np.array([p[1] for p in opts])
    b = {"n_kappa": wl.n_kappa, "n_omega": wl.n_omega, "n_x": wl.n_x, "n_t": wl.n_t,
         "eps": bridge_eps, "max_sum_b2": float(op.sum_b2.max()), "variance": float(var),
         "out_points": [list(p) for p in opts], "u": {}}
    print("bridge plan", time.time() - t0, flush=True)
    for s in SEEDS_BRIDGE:
        C = op.coeffs(s)
        b["u"][str(s)] = [float(v) for v in oracle.field_points(C, wl.n_x, wl.n_t, mx, mt)]
        print("bridge seed", s, time.time() - t0, flush=True)
    out["bridge"] = b

    # large: plan tables and seed-1 coefficients and field at a fixed eps
    wl = W.LARGE
    env = oracle.Envelope("gauss", wl.sigma_g)
    op = oracle.make_plan(spectrum(wl), wl.kappa_u, wl.omega_u, eps=LARGE_EPS, env=env,
                          beta=wl.beta)
    var, m3 = op.moments()
    print("large plan", time.time() - t0, flush=True)
    lpts = lattice_points(wl.n_kappa, wl.n_omega)
    opts = output_points(wl.n_x, wl.n_t)
    mx = np.array([p[0] for p in opts])
    mt = np.array([p[1] for p in opts])
    C = op.coeffs(1)
    q = op.q
    out["large"] = {
        "n_kappa": wl.n_kappa, "n_omega": wl.n_omega, "n_x": wl.n_x, "n_t": wl.n_t,
        "eps": LARGE_EPS, "max_sum_b2": float(op.sum_b2.max()), "variance": float(var),
        "third_moment": float(m3),
        "points": [list(p) for p in lpts],
        "q": [float(q[p]) for p in lpts],
        "sum_b2": [float(op.sum_b2[p]) for p in lpts],
        "coeffs_1": [[[float(C[sh][p].real), float(C[sh][p].imag)] for p in lpts]
                     for sh in range(2)],
        "coeffs_max_abs_1": float(np.abs(C).max()),
        "out_points": [list(p) for p in opts],
        "u_1": [float(v) for v in oracle.field_points(C, wl.n_x, wl.n_t, mx, mt)],
    }
    out["total_seconds"] = time.time() - t0
    with open(os.path.join(HERE, "fields_fullsize.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("done", out["total_seconds"], flush=True)


if __name__ == "__main__":
    main()
