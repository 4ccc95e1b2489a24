"""Writes tests/golden/bridge_256x512.json: expected values for the bridge-span
workload (N_kappa = 256, N_omega = 512, kappa_u = 0.25, omega_u = 4 pi,
U = 40 m/s, z = 20 m, Gaussian envelope sigma_g = 0.25, beta = 0, target
max sum b^2 = 0.5), computed by the FP64 oracle alone:

  * eps from the oracle's bisection (tolerance 1e-13 on max sum b^2),
  * max sum b^2, the exact variance and third moment at that eps,
  * q = S / S_p and sum b^2 at a fixed set of lattice points,
  * C^s_k for seeds 1..4 at the same points, both sheets.

Nothing here comes from the CUDA path.  It takes about an hour on one core
(each bisection step is a full O(N^2) recursion pass; about 45 are needed).

    python tests/golden/make_bridge_golden.py
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

SEEDS = (1, 2, 3, 4)


def sample_points(nk, nw, n_random=56, seed=20231003):
    """Corners, edges and a seeded random spread of lattice points."""
    pts = {(0, 1), (1, 0), (1, 1), (nk - 1, nw - 1), (nk - 1, 1), (1, nw - 1),
           (nk // 2, nw // 2), (nk - 1, nw // 2)}
    rng = np.random.default_rng(seed)
    while len(pts) < 8 + n_random:
        pts.add((int(rng.integers(0, nk)), int(rng.integers(1, nw))))
    return sorted(pts)


def main():
    wl = W.BRIDGE
    oracle.build()
    t0 = time.time()
    S = oracle.kaimal_lorentzian(wl.n_kappa, wl.n_omega, wl.kappa_u, wl.omega_u, wl.U, wl.z,
                                 wl.z0, wl.k_vk, wl.lam)
    env = oracle.Envelope("gauss", wl.sigma_g)
    op = oracle.make_plan(S, wl.kappa_u, wl.omega_u, target=wl.target, env=env, beta=wl.beta)
    t_plan = time.time() - t0
    print("plan", op.eps, t_plan, flush=True)
    var, m3 = op.moments()
    pts = sample_points(wl.n_kappa, wl.n_omega)
    q = op.q
    out = {
        "workload": "bridge_256x512",
        "source": "oracle/ (FP64 bisection, lexicographic recursion, coefficients)",
        "n_kappa": wl.n_kappa, "n_omega": wl.n_omega, "kappa_u": wl.kappa_u,
        "omega_u": wl.omega_u, "U": wl.U, "z": wl.z, "sigma_g": wl.sigma_g,
        "target": wl.target, "beta": wl.beta,
        "eps": op.eps, "max_sum_b2": float(op.sum_b2.max()),
        "variance": float(var), "third_moment": float(m3),
        "points": [list(p) for p in pts],
        "q": [float(q[p]) for p in pts],
        "sum_b2": [float(op.sum_b2[p]) for p in pts],
        "coeffs": {},
        "plan_seconds": t_plan,
    }
    for s in SEEDS:
        C = op.coeffs(s)
        out["coeffs"][str(s)] = [[[float(C[sh][p].real), float(C[sh][p].imag)] for p in pts]
                                 for sh in range(2)]
        out["coeffs_max_abs_" + str(s)] = float(np.abs(C).max())
        print("seed", s, time.time() - t0, flush=True)
    out["total_seconds"] = time.time() - t0
    with open(os.path.join(HERE, "bridge_256x512.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("eps", op.eps, "max_sum_b2", op.sum_b2.max(), "seconds", out["total_seconds"])


if __name__ == "__main__":
    main()
