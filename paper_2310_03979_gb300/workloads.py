"""Seeded synthetic workloads for the SRM3 stochastic-wave hot path.

This module only states inputs: lattice and output sizes, spectrum
parameters, the bispectrum target, seeds and precision.  It holds none of the
method's arithmetic, so both the CUDA path and the FP64 oracle take their
inputs from here.  The random phases of the method are not drawn here: each
side derives them from the per-sample seeds with its own Philox4x32-10.

Spectral model of the workloads (Sec. 5): Kaimal S(omega) with
z0 = 0.03 m and von Karman k = 0.4, times the normalised Lorentzian
wavenumber density a/(pi (a^2 + kappa^2)), a = 7 omega / (2 pi U); bispectrum
|B| = eps g(i,j) sqrt(S_i S_j S_{i+j}) with a Gaussian envelope of width
0.25 of the lattice extent per axis, biphase 0, and eps set so that
max_k sum b_p^2 = target.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    n_kappa: int
    n_omega: int
    kappa_u: float
    omega_u: float
    U: float
    z: float
    n_x: int
    n_t: int
    seeds: tuple
    precision: str = "fp32"          # "fp32" or "fp64"
    storage: str = "auto"            # "auto", "table" or "recompute"
    target: float = 0.5              # max_k sum b_p^2
    sigma_g: float = 0.25
    beta: float = 0.0
    z0: float = 0.03
    k_vk: float = 0.4
    lam: float = 7.0
    # "gauss" (sigma_g), "separable" (g = e(i) e(j) e(i+j), sigma_e) or
    # "sum" (g = b(i+j) alone)
    envelope: str = "gauss"
    sigma_e: float = 0.5
    # fixed bispectrum scale (> 0: used as given, no search on target)
    eps: float = 0.0
    # "sum" (pairs within a sheet) or "mixed" (also the opposite-sign
    # frequency pairs of the general form)
    interactions: str = "sum"

    def envelope_table(self) -> np.ndarray:
        """Separable envelope e(kk, kw) = exp(-1/2 ((kk/(sigma_e Nk))^2 +
        (kw/(sigma_e Nw))^2)), so that g(i, j) = e(i) e(j) e(i+j)."""
        kk = np.arange(self.n_kappa, dtype=np.float64)[:, None] / (self.sigma_e * self.n_kappa)
        kw = np.arange(self.n_omega, dtype=np.float64)[None, :] / (self.sigma_e * self.n_omega)
        return np.exp(-0.5 * (kk * kk + kw * kw))

    def envelope_tables(self):
        """(a, b) with g(i, j) = a(i) a(j) b(i+j); b None means b = a.
        "sum": a = 1 and b(k) = 1 / (2 sqrt((kk + 1/2)(kw + 1/2))), the
        1/sqrt(omega_k kappa_k) shape of the wind-field bispectrum of Sec. 5
        with the lattice points taken at their cell centres."""
        if self.envelope == "separable":
            return self.envelope_table(), None
        if self.envelope == "sum":
            kk = np.arange(self.n_kappa, dtype=np.float64)[:, None] + 0.5
            kw = np.arange(self.n_omega, dtype=np.float64)[None, :] + 0.5
            return np.ones((self.n_kappa, self.n_omega)), 0.5 / np.sqrt(kk * kw)
        raise ValueError(self.envelope)

    @property
    def n_samples(self) -> int:
        return len(self.seeds)

    def with_seeds(self, seeds) -> "Workload":
        return replace(self, seeds=tuple(int(s) for s in seeds))

    def pairs(self) -> int:
        """Unordered pairs sum_k |Pi(k)| of the quadrant lattice."""
        kk = np.arange(self.n_kappa, dtype=np.int64)[:, None]
        kw = np.arange(self.n_omega, dtype=np.int64)[None, :]
        n = (kk + 1) * (kw + 1) - 2
        cnt = (n + 1) // 2
        cnt[0, 0] = 0
        return int(cnt.sum())

    def diff_pairs(self) -> int:
        """Difference (opposite-sign) pairs of one sheet: sum over kw >= 1 of
        (kk + 1)(Nw - 1 - kw); 0 unless interactions == "mixed"."""
        if self.interactions != "mixed":
            return 0
        kk = np.arange(self.n_kappa, dtype=np.int64)[:, None]
        kw = np.arange(1, self.n_omega, dtype=np.int64)[None, :]
        return int(((kk + 1) * (self.n_omega - 1 - kw)).sum())

    def pair_terms_per_sample(self) -> int:
        """One pair-term = one W_ij y_i y_j product for one sheet of one sample."""
        return 2 * (self.pairs() + self.diff_pairs())


# Tiny plain-method case: 32 x 32 lattice, FP64, one sample, 64 x 64 field.
TINY = Workload("tiny_32x32_fp64", 32, 32, 0.5, 4 * math.pi, 30.0, 20.0, 64, 64,
                (1,), precision="fp64", storage="recompute")

# Bridge-span wave: 256 x 512 lattice, stored W table, 64 samples, FP32.
BRIDGE = Workload("bridge_256x512_table_fp32", 256, 512, 0.25, 4 * math.pi, 40.0,
                  20.0, 512, 1024, tuple(range(1, 65)), precision="fp32",
                  storage="table")

# Large grid with W recomputed on the fly: 512 x 1024 lattice, 16 samples.
LARGE = Workload("large_512x1024_recompute_fp32", 512, 1024, 0.25, 4 * math.pi,
                 40.0, 20.0, 1024, 2048, tuple(range(1, 17)), precision="fp32",
                 storage="recompute")

# Profiling case: the bridge spectrum on a 128 x 256 lattice, stored W table
# (0.56 GB, above L2), 64 samples -- two 64-wide sample groups per super-tile
# as in the bridge workload, small enough for multi-pass ncu captures.
PROF128 = Workload("table_128x256_fp32", 128, 256, 0.25, 4 * math.pi, 40.0, 20.0, 256, 512,
                   tuple(range(1, 65)), precision="fp32", storage="table")

# The bridge-span wave with W recomputed from its envelope factors instead of
# stored: the same lattice, samples and seeds, the storage the autotuner picks
# for this shape.
BRIDGE_RC = Workload("bridge_256x512_recompute_fp32", 256, 512, 0.25, 4 * math.pi, 40.0,
                     20.0, 512, 1024, tuple(range(1, 65)), precision="fp32",
                     storage="recompute")

# The bridge-span lattice with a separable envelope g = e(i) e(j) e(i+j)
# (e a Gaussian of width 0.5 of the lattice per axis): the pair sum becomes
# an FFT self-convolution.
BRIDGE_SEP = Workload("bridge_256x512_separable_fp32", 256, 512, 0.25, 4 * math.pi, 40.0,
                      20.0, 512, 1024, tuple(range(1, 65)), precision="fp32",
                      storage="recompute", envelope="separable", sigma_e=0.5)

# The wind field along the long-span bridge of Sec. 5: L = 628 m, omega_u =
# pi rad/s, N_omega = 128, N_t = 2048, N_x = 1024, N_kappa = 256, kappa_u =
# 2 (N_kappa - 1) pi / L; Kaimal with z = 50 m, z0 = 0.03 m, U = 40 m/s,
# k = 0.4; Davenport coherence with lambda = 10, whose wavenumber density
# has half-width lambda omega / (pi U), i.e. lam = 2 lambda = 20 in this
# module's a = lam omega / (2 pi U); 1000 samples, FP32.  Bispectrum of
# Sec. 5: |B| = (2 / (3 sqrt 3)) sqrt(S_i S_j S_k) / sqrt(omega_k kappa_k),
# an envelope of i + j alone, with omega_k kappa_k taken at the cell centres
# ((kk + 1/2) dk (kw + 1/2) dw, the "sum" envelope b(k) = 1 / (2 sqrt((kk +
# 1/2)(kw + 1/2)))), so b_p^2 = eps^2 dk dw b_k^2 q_i q_j matches the paper's
# (2 / (3 sqrt 3))^2 q_i q_j / ((kk + 1/2)(kw + 1/2)) at
# eps = (4 / (3 sqrt 3)) / sqrt(dk dw), a fixed scale (no search).
def _paper_bridge():
    L, nk, nw = 628.0, 256, 128
    ku, wu = 2.0 * (nk - 1) * math.pi / L, math.pi
    eps = (4.0 / (3.0 * math.sqrt(3.0))) / math.sqrt((ku / nk) * (wu / nw))
    return Workload("paper_bridge_256x128_fp32", nk, nw, ku, wu, 40.0, 50.0, 1024, 2048,
                    tuple(range(1, 1001)), precision="fp32", storage="recompute",
                    lam=20.0, envelope="sum", eps=eps)


PAPER_BRIDGE = _paper_bridge()

# The bridge-span wave with the mixed-sign (difference) interactions of the
# general form as well: the same lattice, spectrum, target and seeds, W
# recomputed (about three times the pair-terms of the sum interactions).
BRIDGE_MIXED = Workload("bridge_256x512_mixed_fp32", 256, 512, 0.25, 4 * math.pi, 40.0,
                        20.0, 512, 1024, tuple(range(1, 65)), precision="fp32",
                        storage="recompute", interactions="mixed")

CONFIGS = {"tiny": TINY, "bridge": BRIDGE, "bridge_rc": BRIDGE_RC, "bridge_sep": BRIDGE_SEP,
           "bridge_mixed": BRIDGE_MIXED,
           "large": LARGE, "prof128": PROF128, "paper_bridge": PAPER_BRIDGE}


def uneven_batch(n_spectra: int = 200, seed: int = 4):
    """Uneven batch: spectra with power-of-two grids between 32 and 256 per
    axis, U in [20, 50] m/s, z in [10, 60] m, target in [0.1, 0.7] and 1..32
    samples each (numpy PCG64 with the given seed).  Cutoffs as TINY.
    Sample seeds are 1000 * spectrum_id + j."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.array([32, 64, 128, 256])
    out = []
    for s in range(n_spectra):
        nk = int(rng.choice(sizes))
        nw = int(rng.choice(sizes))
        U = float(rng.uniform(20.0, 50.0))
        z = float(rng.uniform(10.0, 60.0))
        tgt = float(rng.uniform(0.1, 0.7))
        ns = int(rng.integers(1, 33))
        out.append(Workload(f"uneven_{s}", nk, nw, 0.5, 4 * math.pi, U, z, 2 * nk,
                            2 * nw, tuple(1000 * s + j for j in range(ns)),
                            precision="fp32", storage="auto", target=tgt))
    return out


def small_case(nk=24, nw=37, nx=64, nt=128, seeds=(1, 2, 3), precision="fp32",
               storage="recompute", U=30.0, z=20.0, target=0.5, sigma_g=0.25,
               kappa_u=0.5, omega_u=4 * math.pi, beta=0.0) -> Workload:
    """A lattice small enough for the oracle in seconds, ragged against the
    kernels' tiles (neither axis a multiple of 8 by default)."""
    return Workload(f"small_{nk}x{nw}", nk, nw, kappa_u, omega_u, U, z, nx, nt,
                    tuple(seeds), precision=precision, storage=storage,
                    target=target, sigma_g=sigma_g, beta=beta)
