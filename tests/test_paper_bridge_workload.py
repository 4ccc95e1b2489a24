"""The bridge wind field of Sec. 5 as a workload: its grid reproduces the
paper's printed intervals through the FFT-form grid relations (Sec. 4.3), and
its fixed bispectrum scale turns the "sum" envelope into the paper's
bicoherence at the cell centres (the reading of the singular axes)."""
import math

import numpy as np

from paper_2310_03979_gb300 import workloads as W


def test_grid_matches_the_printed_intervals():
    wl = W.PAPER_BRIDGE
    L = 628.0
    dk, dw = wl.kappa_u / wl.n_kappa, wl.omega_u / wl.n_omega
    assert (wl.n_kappa, wl.n_omega, wl.n_x, wl.n_t) == (256, 128, 1024, 2048)
    assert abs(wl.kappa_u - 2.55) < 0.005
    # dk dx = 2 pi / n_x and dw dt = 2 pi / n_t give the printed 0.6135 m and
    # 0.124 s to within the cutoff / N (not N - 1) reading of the spacings:
    # 0.4 % and 0.8 %
    dx, dt = 2 * math.pi / (dk * wl.n_x), 2 * math.pi / (dw * wl.n_t)
    assert abs(dx - L / wl.n_x) / (L / wl.n_x) < 0.005
    assert abs(dx / (L / wl.n_x) - wl.n_kappa / (wl.n_kappa - 1)) < 1e-12
    assert abs(dt - 0.124) / 0.124 < 0.01
    assert (wl.U, wl.z, wl.z0, wl.k_vk) == (40.0, 50.0, 0.03, 0.4)
    assert wl.lam == 20.0  # lambda = 10: half-width lambda omega / (pi U)
    assert wl.n_samples == 1000


def test_fixed_scale_gives_the_papers_bicoherence():
    # b_p^2 = eps^2 dk dw b_k^2 q_i q_j must equal
    # (2 / (3 sqrt 3))^2 q_i q_j / (omega_k kappa_k / (dk dw)) at cell centres
    wl = W.PAPER_BRIDGE
    dk, dw = wl.kappa_u / wl.n_kappa, wl.omega_u / wl.n_omega
    a, b = wl.envelope_tables()
    assert np.all(a == 1.0)
    kk = np.arange(wl.n_kappa)[:, None] + 0.5
    kw = np.arange(wl.n_omega)[None, :] + 0.5
    ours = wl.eps ** 2 * dk * dw * b ** 2
    paper = (2.0 / (3.0 * math.sqrt(3.0))) ** 2 / ((kk * dk) * (kw * dw)) * (dk * dw)
    np.testing.assert_allclose(ours, paper, rtol=1e-13)
