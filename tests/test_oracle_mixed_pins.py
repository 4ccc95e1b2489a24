"""Pins of the oracle's mixed-sign (difference) interactions.

The general form of the method (Eq. truncated_cosines_1d_wave; the mixed
cosines of Eq. quadrant_1d_wave; the signed sums i_w + j_w = +-k_w of
Eq. fft_2d_2_parts) pairs frequencies of opposite sign as well.  The reading
the oracle follows: a point is a signed frequency; the pairs of an output
point k on sheet s are the same-sheet pairs i + j = k of the plain model and
the opposite-sheet pairs whose signed frequencies add up to k's (both parts
off omega = 0, output off omega = 0); the bispectrum is the plain model's
formula at the signed points (Gaussian envelope of the signed frequency
difference); S_p is the largest fixed point of Eq. pure.

Each test checks the oracle against something it does not share: a
hand-solved 1 x 4 lattice, a brute force over all ordered pairs of signed
lattice points (pair set, fixed-point residual, coefficients), closed forms
of the variance and third moment in S and g alone, eps = 0, scale invariance,
the literal cosine series, and a Monte Carlo estimate of the moments.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2310_03979_gb300 import workloads as W


def _gauss(nk, nw, sg):
    def g(ik, iw, jk, jw):  # signed omega indices
        return (math.exp(-0.5 * ((ik - jk) / (sg * nk)) ** 2)
                * math.exp(-0.5 * ((iw - jw) / (sg * nw)) ** 2))
    return g


def _points(nk, nw):
    """Signed lattice points as (sheet, kk, kw): sheet 0 carries +omega,
    sheet 1 carries -omega; the signed frequency index is +-kw."""
    return [(s, a, w) for s in (0, 1) for a in range(nk) for w in range(nw)]


def _sigma(p):
    return p[2] if p[0] == 0 else -p[2]


def _is_pair(P, Q, out):
    """Whether the ordered (P, Q) is a pair of output point `out`."""
    s, kk, kw = out
    if P[1] + Q[1] != kk or _sigma(P) + _sigma(Q) != _sigma(out):
        return False
    if (P[1], P[2]) == (0, 0) or (Q[1], Q[2]) == (0, 0):
        return False
    if P[0] == Q[0]:
        return P[0] == s                      # sum pair on the output's sheet
    return P[2] >= 1 and Q[2] >= 1 and kw >= 1  # difference pair


def _brute_sum_b2(S, Sp, eps, g, dkdw):
    """sum over all pairs of b_p^2, by ordered pairs (off-diagonal halved)."""
    nk, nw = S.shape
    pts = _points(nk, nw)
    out = np.zeros((2, nk, nw))
    for o in pts:
        s, kk, kw = o
        if S[kk, kw] <= 0:
            continue
        tot = dia = 0.0
        for P in pts:
            for Q in pts:
                if not _is_pair(P, Q, o):
                    continue
                Si, Sj = S[P[1], P[2]], S[Q[1], Q[2]]
                B = eps * g(P[1], _sigma(P), Q[1], _sigma(Q)) * math.sqrt(Si * Sj * S[kk, kw])
                if B == 0:
                    continue
                b2 = B * B * dkdw / (Sp[P[1], P[2]] * Sp[Q[1], Q[2]] * S[kk, kw])
                tot += b2
                if P == Q:
                    dia += b2
        out[s, kk, kw] = 0.5 * (tot + dia)
    return out


def _case(nk, nw, U=30.0, z=20.0):
    c = W.small_case(nk=nk, nw=nw, U=U, z=z)
    S = oracle.kaimal_lorentzian(nk, nw, c.kappa_u, c.omega_u, c.U, c.z)
    return c, S


def test_mixed_hand_solved_1x4(oracle_lib):
    """nk = 1, nw = 4, S = (0, 1, 1, 1), dk dw = 1, sigma_g = 1 (g^2 of a
    signed difference d: exp(-d^2 / 16)).  Pairs, written out:
      k = 1: difference {2+, 1-} (d = 3), {3+, 2-} (d = 5)
      k = 2: sum {1, 1} (d = 0), difference {3+, 1-} (d = 4)
      k = 3: sum {1, 2} (d = 1)
    The fixed point q = 1/(1 - sum b^2) solved here by Newton's method."""
    S = np.array([[0.0, 1.0, 1.0, 1.0]])
    eps = 0.3  # past about 0.4 the loop k = 1 -> 2 -> 1 has no fixed point
    Sp, sb2, sweeps = oracle.recursion_mixed(S, 1.0, 4.0, eps, oracle.Envelope("gauss", 1.0))
    G = lambda d: math.exp(-d * d / 16.0)  # noqa: E731
    e2 = eps * eps

    def F(q):
        q1, q2, q3 = q
        return np.array([
            e2 * (G(3) * q2 * q1 + G(5) * q3 * q2),
            e2 * (G(0) * q1 * q1 + G(4) * q3 * q1),
            e2 * (G(1) * q1 * q2)])

    q = np.ones(3)
    for _ in range(200):  # plain fixed point to convergence, then Newton polish
        q = 1.0 / (1.0 - F(q))
    for _ in range(5):
        r = q - 1.0 / (1.0 - F(q))
        h = 1e-7
        Jm = np.zeros((3, 3))
        for c in range(3):
            dq = q.copy()
            dq[c] += h
            Jm[:, c] = ((dq - 1.0 / (1.0 - F(dq))) - r) / h
        q = q - np.linalg.solve(Jm, r)
    x = 1.0 - 1.0 / q
    assert sweeps >= 3
    np.testing.assert_allclose(sb2[0, 1:], x, rtol=1e-13)
    np.testing.assert_allclose(Sp[0, 1:], 1.0 - x, rtol=1e-13)
    assert sb2[0, 0] == 0.0


@pytest.mark.parametrize("nk,nw,eps", [(3, 7, 0.7), (5, 6, 0.8), (1, 9, 0.4)])
def test_mixed_fixed_point_brute_force(oracle_lib, nk, nw, eps):
    """The returned S_p is a fixed point of Eq. pure over the full pair set
    (ordered pairs of signed points by brute force): sum b^2 recomputed from
    it equals the oracle's, on both sheets, to 1e-13."""
    c, S = _case(nk, nw)
    env = oracle.Envelope("gauss", 0.4)
    Sp, sb2, _ = oracle.recursion_mixed(S, c.kappa_u, c.omega_u, eps, env)
    dkdw = (c.kappa_u / nk) * (c.omega_u / nw)
    bf = _brute_sum_b2(S, Sp, eps, _gauss(nk, nw, 0.4), dkdw)
    np.testing.assert_allclose(bf[0], bf[1], rtol=1e-14, atol=0)  # sheets agree
    np.testing.assert_allclose(sb2, bf[0], rtol=1e-13, atol=1e-300)
    np.testing.assert_allclose(Sp, S * (1.0 - bf[0]), rtol=1e-13, atol=1e-300)
    # the difference pairs carry weight here: the plain recursion differs
    Sp0, _ = oracle.recursion(S, c.kappa_u, c.omega_u, eps, env)
    assert np.abs(Sp0 - Sp).max() > 1e-6 * S.max()


def test_mixed_sum_only_equals_plain_recursion(oracle_lib):
    """A lattice one omega step wide has no difference pairs: the fixed point
    is the plain recursion, bit for bit, reached after the second sweep."""
    c, S = _case(6, 2)
    env = oracle.Envelope("gauss", 0.3)
    Sp, sb2, sweeps = oracle.recursion_mixed(S, c.kappa_u, c.omega_u, 2.0, env)
    Sp0, sb0 = oracle.recursion(S, c.kappa_u, c.omega_u, 2.0, env)
    np.testing.assert_array_equal(Sp, Sp0)
    np.testing.assert_array_equal(sb2, sb0)
    assert sweeps == 2


def test_mixed_coeffs_brute_force(oracle_lib):
    """C^s_k with difference pairs equals the brute force over all ordered
    pairs of signed lattice points: pure term plus
    sqrt(S_k) sum b e^{i(phi_P + phi_Q + beta)}, off-diagonal halved."""
    c, S = _case(4, 6)
    nk, nw = S.shape
    env = oracle.Envelope("gauss", 0.4)
    p = oracle.make_plan(S, c.kappa_u, c.omega_u, eps=0.8, env=env, beta=0.35, mixed=True)
    C = p.coeffs(9)
    _, phi = oracle.phases(nk, nw, 9)
    g = _gauss(nk, nw, 0.4)
    dkdw = (c.kappa_u / nk) * (c.omega_u / nw)
    pts = _points(nk, nw)
    for o in pts:
        s, kk, kw = o
        tot = dia = 0j
        if S[kk, kw] > 0:
            for P in pts:
                for Q in pts:
                    if not _is_pair(P, Q, o):
                        continue
                    Si, Sj = S[P[1], P[2]], S[Q[1], Q[2]]
                    B = p.eps * g(P[1], _sigma(P), Q[1], _sigma(Q)) * math.sqrt(Si * Sj * S[kk, kw])
                    if B == 0:
                        continue
                    b = B * math.sqrt(dkdw) / math.sqrt(p.Sp[P[1], P[2]] * p.Sp[Q[1], Q[2]] * S[kk, kw])
                    t = b * np.exp(1j * (phi[P] + phi[Q] + p.beta))
                    tot += t
                    if P == Q:
                        dia += t
        want = 2 * math.sqrt(dkdw) * (math.sqrt(max(p.Sp[kk, kw], 0)) * np.exp(1j * phi[o])
                                      + math.sqrt(S[kk, kw]) * 0.5 * (tot + dia))
        assert abs(C[o] - want) <= 1e-12 * max(1.0, abs(want)), o


def test_mixed_moments_closed_form(oracle_lib):
    """Variance identity var = 4 dk dw sum S (S_p takes up exactly the power
    the difference pairs carry) and E[u^3] = sum over every pair, both
    sheets, of m 2 eps g (dk dw)^2 sqrt(S_i S_j S_k) cos(beta) (m = 3 on the
    diagonal, else 6), in S and g alone."""
    c, S = _case(4, 7)
    nk, nw = S.shape
    env = oracle.Envelope("gauss", 0.4)
    p = oracle.make_plan(S, c.kappa_u, c.omega_u, eps=0.75, env=env, beta=0.25, mixed=True)
    var, m3 = p.moments()
    dkdw = (c.kappa_u / nk) * (c.omega_u / nw)
    assert var == pytest.approx(4 * dkdw * S.sum(), rel=1e-13)
    g = _gauss(nk, nw, 0.4)
    pts = _points(nk, nw)
    tot = 0.0
    for o in pts:
        for P in pts:
            for Q in pts:
                if not _is_pair(P, Q, o):
                    continue
                B = p.eps * g(P[1], _sigma(P), Q[1], _sigma(Q)) * math.sqrt(
                    S[P[1], P[2]] * S[Q[1], Q[2]] * S[o[1], o[2]])
                # ordered pairs: each off-diagonal pair twice (weight 6 / 2)
                tot += (3.0 if P == Q else 3.0) * 2 * dkdw ** 2 * B * math.cos(p.beta)
    assert m3 == pytest.approx(tot, rel=1e-12)
    p0 = oracle.make_plan(S, c.kappa_u, c.omega_u, eps=0.75, env=env, beta=0.25)
    assert abs(m3 - p0.moments()[1]) > 1e-3 * abs(m3)  # the difference triples count


def test_mixed_eps_zero_and_scale_invariance(oracle_lib):
    c, S = _case(5, 8)
    env = oracle.Envelope("gauss", 0.4)
    Sp, sb2, _ = oracle.recursion_mixed(S, c.kappa_u, c.omega_u, 0.0, env)
    np.testing.assert_array_equal(Sp, S)
    assert not sb2.any()
    Sp1, _, _ = oracle.recursion_mixed(S, c.kappa_u, c.omega_u, 0.75, env)
    Sp2, _, _ = oracle.recursion_mixed(7.5 * S, c.kappa_u, c.omega_u, 0.75, env)
    np.testing.assert_allclose(Sp2, 7.5 * Sp1, rtol=1e-13)


def test_mixed_series_equals_fft_form(oracle_lib):
    """The literal cosine series with the mixed cosines, each written at the
    frequencies of its two parts, equals coefficients + DFT."""
    c = W.small_case(nk=4, nw=6, nx=8, nt=16)
    S = oracle.kaimal_lorentzian(c.n_kappa, c.n_omega, c.kappa_u, c.omega_u, c.U, c.z)
    env = oracle.Envelope("gauss", 0.4)
    p = oracle.make_plan(S, c.kappa_u, c.omega_u, eps=0.8, env=env, beta=0.4, mixed=True)
    u = p.field(3, c.n_x, c.n_t)
    mx, mt = np.meshgrid(np.arange(c.n_x), np.arange(c.n_t), indexing="ij")
    us = oracle.field_series(S, p.Sp, c.kappa_u, c.omega_u, p.eps, 3, c.n_x, c.n_t,
                             mx.ravel(), mt.ravel(), env, p.beta, mixed=True)
    sig = math.sqrt(p.moments()[0])
    np.testing.assert_allclose(us.reshape(u.shape), u, rtol=0, atol=1e-11 * sig)


def test_mixed_bisection_reaches_target(oracle_lib):
    c, S = _case(4, 8)
    env = oracle.Envelope("gauss", 0.4)
    eps, mx, _, Sp, sb2 = oracle.bisect_eps(S, c.kappa_u, c.omega_u, 0.5, env, mixed=True)
    assert abs(mx - 0.5) <= 1e-13
    Sp2, sb22, _ = oracle.recursion_mixed(S, c.kappa_u, c.omega_u, eps, env)
    np.testing.assert_array_equal(Sp, Sp2)
    eps0, _, _, _, _ = oracle.bisect_eps(S, c.kappa_u, c.omega_u, 0.5, env)
    assert eps < eps0  # the difference pairs take up part of the budget


def test_mixed_monte_carlo_moments(oracle_lib):
    """Sample variance and third moment over many seeds match the exact
    moments of the mixed model within 5 standard errors."""
    c = W.small_case(nk=3, nw=5, nx=4, nt=16)
    S = oracle.kaimal_lorentzian(c.n_kappa, c.n_omega, c.kappa_u, c.omega_u, c.U, c.z)
    env = oracle.Envelope("gauss", 0.5)
    p = oracle.make_plan(S, c.kappa_u, c.omega_u, target=0.6, env=env, mixed=True)
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
    assert m3 > 10 * se3
