"""Failure detection without a GPU fault: the bounded waits of the recursion's
grid barrier and of the FP32 pair sum's mbarrier pipeline give up, raise their
error words and return (srm3_selftest_timeouts), and the device stays usable:
a plan built and sampled afterwards still matches the oracle."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2310_03979_gb300 import srm3
from paper_2310_03979_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_waits_time_out_and_the_context_survives(oracle_lib):
    bar, wait = ctypes.c_int(-1), ctypes.c_int(-1)
    assert srm3.load().srm3_selftest_timeouts(ctypes.byref(bar), ctypes.byref(wait)) == 0
    assert bar.value == 1 and wait.value == 1
    wl = W.small_case(nk=24, nw=37, nx=64, nt=128, seeds=(3,), precision="fp32")
    S = oracle.kaimal_lorentzian(wl.n_kappa, wl.n_omega, wl.kappa_u, wl.omega_u, wl.U, wl.z)
    op = oracle.make_plan(S, wl.kappa_u, wl.omega_u, target=wl.target,
                          env=oracle.Envelope("gauss", wl.sigma_g))
    with srm3.Plan.create(wl) as p:
        u = p.sample([3]).cpu().numpy()[0]
    ref = op.field(3, wl.n_x, wl.n_t)
    assert np.abs(u - ref).max() <= 1e-4 * math.sqrt(op.moments()[0])
