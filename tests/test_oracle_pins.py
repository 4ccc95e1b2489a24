"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test checks the oracle against something the paper or mathematics fixes:
a hand-worked recursion, a library routine (cuRAND's host Philox, numpy's
FFT), a reduction to the 2nd-order SRM, a closed-form integral, or Monte Carlo
moments of the series.
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

import oracle
from paper_2310_03979_gb300 import workloads as W


# --------------------------------------------------------------------------
# Spectrum (Sec. 5)

def test_kaimal_integral_closed_form(oracle_lib):
    """The Kaimal spectrum integrates to 3 u*^2 on (0, inf) per sheet,
    i.e. sigma_u^2 = 6 u*^2 over both signs of omega (the textbook Kaimal
    normalisation).  The partial integral has the closed form
    3 u*^2 [(1 + c w_a)^(-2/3) - (1 + c w_b)^(-2/3)], c = 50 z / (2 pi U)."""
    U, z = 35.0, 25.0
    nw, omega_u = 40001, 40.0
    S = oracle.kaimal_lorentzian(1, nw, 1.0, omega_u, U, z)[0]
    dw = omega_u / nw
    omega = np.arange(nw) * dw
    a = 7.0 * omega / (2 * math.pi * U)
    kaimal = S[1:] * math.pi * a[1:]           # Lorentzian peak is 1/(pi a)
    from scipy.integrate import simpson
    num = simpson(kaimal, x=omega[1:])
    ustar = 0.4 * U / math.log(z / 0.03)
    c = 50 * z / (2 * math.pi * U)
    closed = 3 * ustar ** 2 * ((1 + c * omega[1]) ** (-2 / 3) - (1 + c * omega[-1]) ** (-2 / 3))
    assert abs(num - closed) / closed < 1e-8
    assert np.all(S[0] == 0.0)                  # omega = 0 column is zero


def test_lorentzian_half_width(oracle_lib):
    """a/(pi(a^2+kappa^2)) halves at kappa = a: choose dk = 7 dw / (2 pi U)
    so that a(omega_m) is the lattice wavenumber kappa_m."""
    U, nk, nw, omega_u = 30.0, 16, 16, 4 * math.pi
    dw = omega_u / nw
    dk = 7 * dw / (2 * math.pi * U)
    S = oracle.kaimal_lorentzian(nk, nw, nk * dk, omega_u, U, 20.0)
    for m in range(1, nk):
        assert S[m, m] / S[0, m] == pytest.approx(0.5, rel=1e-13)
    assert S[0, 0] == 0.0


# --------------------------------------------------------------------------
# Philox4x32-10 against cuRAND's host generator (a library)

def _curand():
    cands = [ctypes.util.find_library("curand"), "/usr/local/cuda/lib64/libcurand.so",
             "libcurand.so.10"]
    for c in cands:
        if not c:
            continue
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def _curand_host_words(lib, seed, n):
    gen = ctypes.c_void_p()
    PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


def test_philox_matches_curand_host(oracle_lib):
    """cuRAND's host Philox4_32_10 (default ordering) emits, as its first
    blocks, Philox4x32-10 at counter (0, 0, b, 0) under key = (seed lo, seed hi)."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    for seed in (1, 2, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF):
        ref = _curand_host_words(lib, seed, 4 * 64).reshape(64, 4)
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
        for b in range(64):
            got = oracle.philox4x32_10(np.array([0, 0, b, 0], dtype=np.uint32), key)
            assert np.array_equal(got, ref[b]), (seed, b)


def test_phase_counter_map(oracle_lib):
    """Phase word of (sheet s, kk, kw) is lane e & 3 of Philox at counter
    e >> 2 (low word first), e = (s Nk + kk) Nw + kw; phi = 2 pi (w + 1/2) 2^-32."""
    nk, nw, seed = 5, 7, 0xDEADBEEF12
    words, phi = oracle.phases(nk, nw, seed)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    for s in range(2):
        for kk in range(nk):
            for kw in range(nw):
                e = (s * nk + kk) * nw + kw
                blk = oracle.philox4x32_10(np.array([e >> 2, 0, 0, 0], dtype=np.uint32), key)
                assert words[s, kk, kw] == blk[e & 3]
    assert np.all(phi > 0) and np.all(phi < 2 * math.pi)
    np.testing.assert_array_equal(phi, 2 * math.pi * ((words.astype(np.float64) + 0.5) * 2.0 ** -32))


# --------------------------------------------------------------------------
# Recursion (Eq. pure)

def test_recursion_hand_worked_3x3(oracle_lib):
    """3 x 3 lattice, S = 1 except S(0,0) = 0, dk = dw = 1, Gaussian
    envelope with sigma_g = 0.5 (1.5 lattice steps): G(d) = exp(-d^2/4.5).
    The canonical pairs and the recursion written out by hand."""
    S = np.ones((3, 3))
    S[0, 0] = 0.0
    eps = 0.3
    Sp, sb2 = oracle.recursion(S, 3.0, 3.0, eps, oracle.Envelope("gauss", 0.5))
    G = lambda d: math.exp(-d * d / 4.5)
    e2 = eps * eps
    x = {}
    x[(0, 1)] = 0.0
    x[(1, 0)] = 0.0
    x[(0, 2)] = e2                                 # {(0,1),(0,1)}
    x[(2, 0)] = e2                                 # {(1,0),(1,0)}
    x[(1, 1)] = e2 * G(1) ** 4                     # {(0,1),(1,0)}
    q = lambda k: 1.0 / (1.0 - x[k])
    x[(1, 2)] = e2 * G(1) ** 2 * q((1, 1)) + e2 * G(1) ** 2 * G(2) ** 2 * q((0, 2))
    x[(2, 1)] = e2 * G(1) ** 2 * G(2) ** 2 * q((2, 0)) + e2 * G(1) ** 2 * q((1, 1))
    x[(2, 2)] = (e2 * G(2) ** 2 * q((2, 1)) + e2 * G(2) ** 4 * q((0, 2)) * q((2, 0))
                 + e2 * G(2) ** 2 * q((1, 2)) + e2 * q((1, 1)) ** 2)
    assert sb2[0, 0] == 0.0 and Sp[0, 0] == 0.0
    for k, v in x.items():
        assert sb2[k] == pytest.approx(v, rel=1e-14, abs=1e-300), k
        assert Sp[k] == pytest.approx(1.0 - v, rel=1e-14), k


def _sep_setup(nk=7, nw=9, seed=3):
    rng = np.random.default_rng(seed)
    S = oracle.kaimal_lorentzian(nk, nw, 0.5, 4 * math.pi, 30.0, 20.0)
    e = rng.uniform(0.5, 1.5, size=(nk, nw))
    return S, e


def _self_conv_half(v):
    """sum over unordered {i, j}, i + j = k of v_i v_j via a zero-padded
    FFT: (v * v)(k)/2 plus half the diagonal term v_{k/2}^2."""
    nk, nw = v.shape
    F = np.fft.fft2(v, s=(2 * nk, 2 * nw))
    full = np.fft.ifft2(F * F)[:nk, :nw]
    diag = np.zeros((nk, nw), dtype=v.dtype)
    diag[::2, ::2] = v[: (nk + 1) // 2, : (nw + 1) // 2] ** 2
    return 0.5 * (full + diag)


def test_recursion_separable_fft(oracle_lib):
    """With g = e(i) e(j) e(k): sum_b2(k) = eps^2 dk dw e_k^2 [S_k > 0]
    * sum_{Pi(k)} v_i v_j with v = e^2 q [S > 0]; the pair sum computed by a
    zero-padded FFT self-convolution (numpy) from the oracle's own q."""
    S, e = _sep_setup()
    nk, nw = S.shape
    ku, wu, eps = 0.5, 4 * math.pi, 0.15
    env = oracle.Envelope("separable", table=e)
    Sp, sb2 = oracle.recursion(S, ku, wu, eps, env)
    pos = S > 0
    q = np.where(pos, S / np.where(pos, Sp, 1.0), 1.0)
    v = np.where(pos, e * e * q, 0.0)
    half = _self_conv_half(v).real
    pred = eps ** 2 * (ku / nk) * (wu / nw) * e ** 2 * half * pos
    assert sb2.max() > 0.05
    np.testing.assert_allclose(sb2, pred, rtol=1e-11, atol=1e-14 * sb2.max())


def test_recursion_scale_invariance_and_monotone(oracle_lib):
    """S -> c S leaves q and the bisected eps unchanged; max sum_b2 grows
    strictly with eps (which justifies bisection)."""
    c = W.small_case(nk=9, nw=11)
    S = oracle.kaimal_lorentzian(c.n_kappa, c.n_omega, c.kappa_u, c.omega_u, c.U, c.z)
    p1 = oracle.make_plan(S, c.kappa_u, c.omega_u, target=0.5)
    p2 = oracle.make_plan(7.5 * S, c.kappa_u, c.omega_u, target=0.5)
    assert p2.eps == pytest.approx(p1.eps, rel=1e-12)
    np.testing.assert_allclose(p2.q, p1.q, rtol=1e-12)
    assert abs(p1.sum_b2.max() - 0.5) <= 1e-13
    last = -1.0
    for eps in np.linspace(0.0, p1.eps * 1.02, 12):
        _, sb2 = oracle.recursion(S, c.kappa_u, c.omega_u, float(eps))
        assert sb2.max() > last
        last = sb2.max()
    with pytest.raises(oracle.OracleError):
        oracle.recursion(S, c.kappa_u, c.omega_u, p1.eps * 3.0)


# --------------------------------------------------------------------------
# Coefficients and field (Sec. 3 and Sec. 4.3)

def _z(nk, nw, seed):
    _, phi = oracle.phases(nk, nw, seed)
    return np.exp(1j * phi)


def test_coeffs_separable_fft(oracle_lib):
    """Pair part of C^s_k for g = e(i) e(j) e(k) equals
    2 eps dk dw sqrt(S_k) e_k e^{i beta} sum_{Pi(k)} w_i w_j with
    w = e sqrt(q) z [S > 0], the pair sum by numpy FFT self-convolution."""
    S, e = _sep_setup(nk=6, nw=10, seed=5)
    nk, nw = S.shape
    ku, wu, eps, beta, seed = 0.5, 4 * math.pi, 0.05, 0.37, 11
    env = oracle.Envelope("separable", table=e)
    Sp, _ = oracle.recursion(S, ku, wu, eps, env)
    C = oracle.coeffs(S, Sp, ku, wu, eps, seed, env, beta)
    z = _z(nk, nw, seed)
    dkdw = (ku / nk) * (wu / nw)
    pos = S > 0
    q = np.where(pos, S / np.where(pos, Sp, 1.0), 1.0)
    for s in range(2):
        pure = 2 * np.sqrt(dkdw * np.maximum(Sp, 0)) * z[s]
        w = np.where(pos, e * np.sqrt(q) * z[s], 0)
        pair = 2 * eps * dkdw * np.sqrt(S) * e * np.exp(1j * beta) * _self_conv_half(w) * pos
        np.testing.assert_allclose(C[s], pure + pair, rtol=0, atol=1e-12 * np.abs(C[s]).max())


def test_coeffs_ordered_pair_brute_force(oracle_lib):
    """Canonical-half pair sum equals half the sum over all ordered (i, j)
    with i + j = k (i, j != 0) plus half the diagonal, Gaussian envelope."""
    c = W.small_case(nk=5, nw=6)
    S = oracle.kaimal_lorentzian(c.n_kappa, c.n_omega, c.kappa_u, c.omega_u, c.U, c.z)
    p = oracle.make_plan(S, c.kappa_u, c.omega_u, target=0.5)
    nk, nw = S.shape
    dkdw = (c.kappa_u / nk) * (c.omega_u / nw)
    C = p.coeffs(7)
    z = _z(nk, nw, 7)
    Sp = p.Sp
    env = lambda ik, iw, jk, jw: (math.exp(-0.5 * ((ik - jk) / (0.25 * nk)) ** 2)
                                  * math.exp(-0.5 * ((iw - jw) / (0.25 * nw)) ** 2))
    for s in range(2):
        for kk in range(nk):
            for kw in range(nw):
                tot = 0j
                dia = 0j
                if S[kk, kw] > 0:
                    for ik in range(kk + 1):
                        for iw in range(kw + 1):
                            jk, jw = kk - ik, kw - iw
                            if (ik, iw) == (0, 0) or (jk, jw) == (0, 0):
                                continue
                            if S[ik, iw] <= 0 or S[jk, jw] <= 0:
                                continue
                            B = p.eps * env(ik, iw, jk, jw) * math.sqrt(S[ik, iw] * S[jk, jw] * S[kk, kw])
                            b = B * math.sqrt(dkdw) / math.sqrt(Sp[ik, iw] * Sp[jk, jw] * S[kk, kw])
                            t = b * z[s, ik, iw] * z[s, jk, jw]
                            tot += t
                            if (ik, iw) == (jk, jw):
                                dia += t
                pair = 0.5 * (tot + dia)
                want = 2 * math.sqrt(dkdw) * (math.sqrt(max(Sp[kk, kw], 0)) * z[s, kk, kw]
                                              + math.sqrt(S[kk, kw]) * pair)
                assert abs(C[s, kk, kw] - want) <= 1e-12 * max(1.0, abs(want))


def test_field_dft_matches_numpy_fft(oracle_lib):
    """u = Re sum_s sum_k C^s_k e^{i(2pi kk mx/Nx + s 2pi kw mt/Nt)}: the
    oracle's direct sum vs numpy's inverse FFT of the packed spectrum."""
    rng = np.random.default_rng(0)
    nk, nw, nx, nt = 6, 9, 16, 32
    C = rng.normal(size=(2, nk, nw)) + 1j * rng.normal(size=(2, nk, nw))
    u = oracle.field_dft(C, nx, nt)
    F = np.zeros((nx, nt), dtype=complex)
    for kk in range(nk):
        for kw in range(nw):
            F[kk, kw] += C[0, kk, kw]
            F[kk, (-kw) % nt] += C[1, kk, kw]
    ref = np.real(np.fft.ifft2(F)) * nx * nt
    np.testing.assert_allclose(u, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    mx = rng.integers(0, nx, 40)
    mt = rng.integers(0, nt, 40)
    np.testing.assert_allclose(oracle.field_points(C, nx, nt, mx, mt), ref[mx, mt],
                               rtol=0, atol=1e-12 * np.abs(ref).max())


def test_eps_zero_is_second_order_srm(oracle_lib):
    """eps = 0 gives the 2nd-order SRM wave of Sec. 3,
    u = 2 sum_k sum_{+-} sqrt(S dk dw) cos(kappa x +- omega t + phi^{+-}),
    with the same phases (the identical-phase comparison of Sec. 5)."""
    c = W.small_case(nk=6, nw=8, nx=16, nt=32)
    S = oracle.kaimal_lorentzian(c.n_kappa, c.n_omega, c.kappa_u, c.omega_u, c.U, c.z)
    p = oracle.make_plan(S, c.kappa_u, c.omega_u, eps=0.0)
    np.testing.assert_array_equal(p.Sp, S)
    u = p.field(5, c.n_x, c.n_t)
    _, phi = oracle.phases(c.n_kappa, c.n_omega, 5)
    dk, dw = c.kappa_u / c.n_kappa, c.omega_u / c.n_omega
    x = np.arange(c.n_x) * 2 * math.pi / (c.n_x * dk)
    t = np.arange(c.n_t) * 2 * math.pi / (c.n_t * dw)
    ref = np.zeros((c.n_x, c.n_t))
    for kk in range(c.n_kappa):
        for kw in range(c.n_omega):
            a = 2 * math.sqrt(S[kk, kw] * dk * dw)
            ref += a * np.cos(kk * dk * x[:, None] + kw * dw * t[None, :] + phi[0, kk, kw])
            ref += a * np.cos(kk * dk * x[:, None] - kw * dw * t[None, :] + phi[1, kk, kw])
    np.testing.assert_allclose(u, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_series_equals_fft_form(oracle_lib):
    """The literal cosine series (Eq. quadrant_1d_wave, sum interactions)
    equals coefficients + DFT (the FFT form of Sec. 4.3) at every point."""
    c = W.small_case(nk=6, nw=7, nx=16, nt=16)
    S = oracle.kaimal_lorentzian(c.n_kappa, c.n_omega, c.kappa_u, c.omega_u, c.U, c.z)
    p = oracle.make_plan(S, c.kappa_u, c.omega_u, target=0.5, beta=0.4)
    u = p.field(3, c.n_x, c.n_t)
    mx, mt = np.meshgrid(np.arange(c.n_x), np.arange(c.n_t), indexing="ij")
    us = oracle.field_series(S, p.Sp, c.kappa_u, c.omega_u, p.eps, 3, c.n_x, c.n_t,
                             mx.ravel(), mt.ravel(), p.env, p.beta)
    sig = math.sqrt(p.moments()[0])
    np.testing.assert_allclose(us.reshape(u.shape), u, rtol=0, atol=1e-11 * sig)


# --------------------------------------------------------------------------
# Moments

def test_exact_variance_and_third_moment_closed_forms(oracle_lib):
    """var = sum_s sum_k 2 S_k dk dw (pure + pair split of Eq. pure) and
    E[u^3] = sum_s sum_k sum_{Pi(k)} m_ij 2 (dk dw)^2 Re B(i,j), m = 6 or 3."""
    c = W.small_case(nk=6, nw=7)
    S = oracle.kaimal_lorentzian(c.n_kappa, c.n_omega, c.kappa_u, c.omega_u, c.U, c.z)
    p = oracle.make_plan(S, c.kappa_u, c.omega_u, target=0.5, beta=0.3)
    var, m3 = p.moments()
    nk, nw = S.shape
    dkdw = (c.kappa_u / nk) * (c.omega_u / nw)
    assert var == pytest.approx(2 * 2 * dkdw * S.sum(), rel=1e-13)
    tot = 0.0
    for kk in range(nk):
        for kw in range(nw):
            for ik in range(kk + 1):
                for iw in range(kw + 1):
                    jk, jw = kk - ik, kw - iw
                    if (ik, iw) == (0, 0) or (jk, jw) == (0, 0):
                        continue
                    if not (ik < jk or (ik == jk and iw <= jw)):
                        continue
                    g = (math.exp(-0.5 * ((ik - jk) / (0.25 * nk)) ** 2)
                         * math.exp(-0.5 * ((iw - jw) / (0.25 * nw)) ** 2))
                    B = p.eps * g * math.sqrt(S[ik, iw] * S[jk, jw] * S[kk, kw])
                    m = 3 if (ik, iw) == (jk, jw) else 6
                    tot += m * 2 * dkdw ** 2 * B * math.cos(p.beta)
    assert m3 == pytest.approx(2 * tot, rel=1e-12)


def test_monte_carlo_moments(oracle_lib):
    """Sample variance and third moment of the oracle's fields over many
    seeds match the exact ensemble moments (the discrete analogue of the
    paper's skewness validation, Sec. 5): within 5 standard errors, with a
    third moment at least 15 standard errors from zero."""
    c = W.small_case(nk=4, nw=5, nx=8, nt=16)
    S = oracle.kaimal_lorentzian(c.n_kappa, c.n_omega, c.kappa_u, c.omega_u, c.U, c.z)
    p = oracle.make_plan(S, c.kappa_u, c.omega_u, target=0.6)
    var, m3 = p.moments()
    n = 12000
    m2s = np.empty(n)
    m3s = np.empty(n)
    for i in range(n):
        u = p.field(1 + i, c.n_x, c.n_t)
        m2s[i] = np.mean(u * u)
        m3s[i] = np.mean(u ** 3)
    se2 = m2s.std(ddof=1) / math.sqrt(n)
    se3 = m3s.std(ddof=1) / math.sqrt(n)
    assert abs(m2s.mean() - var) < 5 * se2
    assert abs(m3s.mean() - m3) < 5 * se3
    assert m3 > 15 * se3


def test_pair_counts(oracle_lib):
    """|Pi(k)| = ceil(((kk+1)(kw+1) - 2)/2) by brute force, and the
    totals of the three fixed workloads."""
    for nk, nw in [(1, 1), (3, 4), (5, 2), (6, 7)]:
        tot = 0
        for kk in range(nk):
            for kw in range(nw):
                for ik in range(kk + 1):
                    for iw in range(kw + 1):
                        jk, jw = kk - ik, kw - iw
                        if (ik, iw) == (0, 0) or (jk, jw) == (0, 0):
                            continue
                        if ik < jk or (ik == jk and iw <= jw):
                            tot += 1
        wl = W.small_case(nk=nk, nw=nw)
        assert wl.pairs() == tot
    assert W.TINY.pairs() == 138496
    assert abs(W.BRIDGE.pairs() - 2.16e9) / 2.16e9 < 0.01
    assert abs(W.LARGE.pairs() - 3.45e10) / 3.45e10 < 0.01


def test_two_table_separable_recursion_and_coeffs_fft(oracle_lib):
    """g = a(i) a(j) b(i+j): sum_b2(k) = eps^2 dk dw b_k^2 [S_k > 0] sum_{Pi(k)}
    v_i v_j with v = a^2 q [S > 0], and the pair part of C^s_k is
    2 eps dk dw sqrt(S_k) b_k e^{i beta} sum_{Pi(k)} w_i w_j with
    w = a sqrt(q) z [S > 0]; both pair sums by numpy FFT self-convolution.
    b is not a multiple of a, so a swapped or dropped table fails."""
    S, a = _sep_setup(nk=7, nw=9, seed=13)
    nk, nw = S.shape
    rng = np.random.default_rng(21)
    b = 0.3 + rng.random((nk, nw))
    ku, wu, eps, beta, seed = 0.5, 4 * math.pi, 0.07, -0.4, 5
    env = oracle.Envelope("separable", table=a, table_b=b)
    Sp, sb2 = oracle.recursion(S, ku, wu, eps, env)
    pos = S > 0
    q = np.where(pos, S / np.where(pos, Sp, 1.0), 1.0)
    dkdw = (ku / nk) * (wu / nw)
    v = np.where(pos, a * a * q, 0.0)
    pred = eps ** 2 * dkdw * b ** 2 * _self_conv_half(v).real * pos
    assert sb2.max() > 0.01
    np.testing.assert_allclose(sb2, pred, rtol=1e-11, atol=1e-14 * sb2.max())
    C = oracle.coeffs(S, Sp, ku, wu, eps, seed, env, beta)
    z = _z(nk, nw, seed)
    for s in range(2):
        pure = 2 * np.sqrt(dkdw * np.maximum(Sp, 0)) * z[s]
        w = np.where(pos, a * np.sqrt(q) * z[s], 0)
        pair = 2 * eps * dkdw * np.sqrt(S) * b * np.exp(1j * beta) * _self_conv_half(w) * pos
        np.testing.assert_allclose(C[s], pure + pair, rtol=0, atol=1e-12 * np.abs(C[s]).max())
