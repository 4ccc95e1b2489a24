"""Separable envelopes g(i, j) = a(i) a(j) b(i+j) -- one table (a = b = e,
envelope "separable") or an envelope of i + j alone (a = 1, envelope "sum",
the shape of the wind-field bispectrum of Sec. 5): the recursion with the
envelope factors carried on h = a^2 q and b_k^2, and the pair sum as a
zero-padded FFT self-convolution, against the FP64 oracle's O(N^2) sums for
the same envelope (the oracle's separable forms are pinned to a numpy FFT
convolution in test_oracle_pins.py).

Tolerances as in test_gpu_parity.py: FP64 fields 1e-10 sigma_u, FP32 fields
1e-4 sigma_u; FP64 coefficients 1e-11 of max|C|; plan
tables 1e-11 (FP64 plans) and 2e-8 (FP32 plans, eps to 1e-9 of the target);
FP32 coefficients 1e-5 of max|C| (FFT rounding, see the test).
"""
import dataclasses
import functools
import math

import numpy as np
import pytest

import oracle
from paper_2310_03979_gb300 import srm3
from paper_2310_03979_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sep_case(nk=24, nw=37, nx=64, nt=128, seeds=(1, 2, 3), precision="fp64", sigma_e=0.5,
             envelope="separable"):
    wl = W.small_case(nk=nk, nw=nw, nx=nx, nt=nt, seeds=seeds, precision=precision)
    return dataclasses.replace(wl, envelope=envelope, sigma_e=sigma_e,
                               name=f"{envelope}_{nk}x{nw}")


@functools.lru_cache(maxsize=None)
def oracle_plan(wl, eps=None):
    S = oracle.kaimal_lorentzian(wl.n_kappa, wl.n_omega, wl.kappa_u, wl.omega_u, wl.U, wl.z,
                                 wl.z0, wl.k_vk, wl.lam)
    a, b = wl.envelope_tables()
    env = oracle.Envelope("separable", table=a, table_b=b)
    if eps is None:
        return oracle.make_plan(S, wl.kappa_u, wl.omega_u, target=wl.target, env=env,
                                beta=wl.beta)
    return oracle.make_plan(S, wl.kappa_u, wl.omega_u, eps=eps, env=env, beta=wl.beta)


def _cplx(C):
    C = C.cpu().numpy()
    return C[..., 0] + 1j * C[..., 1]


@pytest.mark.parametrize("precision,envelope", [("fp64", "separable"), ("fp32", "separable"),
                                                ("fp64", "sum"), ("fp32", "sum")])
def test_separable_plan_tables_and_eps(oracle_lib, precision, envelope):
    wl = sep_case(precision=precision, envelope=envelope)
    op = oracle_plan(wl)
    with srm3.Plan.create(wl) as p:
        S, q, sb2 = p.tables()
        info = p.info()
    tol, rel = (1e-13, 1e-11) if precision == "fp64" else (1e-9, 2e-8)
    np.testing.assert_allclose(S, op.S, rtol=1e-13, atol=0)
    assert info.eps == pytest.approx(op.eps, rel=rel)
    assert abs(info.max_sum_b2 - wl.target) <= tol
    np.testing.assert_allclose(q, op.q, rtol=rel)
    np.testing.assert_allclose(sb2, op.sum_b2, rtol=rel, atol=1e-15)


@pytest.mark.parametrize("envelope", ["separable", "sum"])
def test_separable_eps_search_coarse_start(envelope):
    """A 256 x 256 lattice with a separable envelope: the eps search starts
    from the root on the 64 x 64 lattice of every fourth point (the factors
    a^2 and b^2 taken at those points), and the FP32 plan's eps agrees with
    the FP64 plan's (target to 1e-13, FP64 passes to the end) to 2e-8."""
    res = {}
    for precision in ("fp64", "fp32"):
        wl = sep_case(nk=256, nw=256, nx=256, nt=512, seeds=(1,), precision=precision,
                      envelope=envelope)
        with srm3.Plan.create(wl) as p:
            res[precision] = p.info()
    for info in res.values():
        assert (info.coarse_fk, info.coarse_fw) == (4, 4)
        # the smooth Gaussian factors place the coarse root inside the window;
        # the sum envelope's b ~ 1/sqrt(kk kw) weights the lattice's lowest
        # points, where the coarse quadrature differs most (either way of the
        # search is correct)
        if envelope == "separable":
            assert info.recursion_flags & srm3.SRM3_REC_COARSE_START
    assert abs(res["fp64"].max_sum_b2 - wl.target) <= 1e-13
    assert abs(res["fp32"].max_sum_b2 - wl.target) <= 1e-9
    assert res["fp32"].eps == pytest.approx(res["fp64"].eps, rel=2e-8)


@pytest.mark.parametrize("nk,nw", [(24, 37), (40, 70), (1, 9), (9, 1), (100, 180)])
def test_separable_recursion_at_fixed_eps(oracle_lib, nk, nw):
    """The bulk of a separable pass is an online FFT self-convolution of h
    (levels 16 and up); its rounding is bounded norm-wise, |ds_k| <~ u
    log2(N) sum_i h_i^2, about 1e-14 of the largest pair sum here, hence an
    absolute term of 1e-13 max(sum_b2) beside the relative one."""
    pow2 = lambda n: 1 << max(1, (2 * n - 1).bit_length())  # noqa: E731
    wl = sep_case(nk=nk, nw=nw, nx=pow2(nk), nt=pow2(nw))
    eps = 1.5 if nk > 1 and nw > 1 else 0.5  # max sum_b2 0.2 - 0.3 on the 2-D lattices
    op = oracle_plan(wl, eps=eps)
    with srm3.Plan.create(wl, eps=eps) as p:
        _, q, sb2 = p.tables()
    np.testing.assert_allclose(q, op.q, rtol=1e-13)
    np.testing.assert_allclose(sb2, op.sum_b2, rtol=1e-13, atol=1e-13 * op.sum_b2.max())


@pytest.mark.parametrize("precision,nk,nw,beta,envelope", [
    ("fp64", 24, 37, 0.0, "separable"), ("fp32", 24, 37, 0.0, "separable"),
    ("fp64", 40, 70, 0.6, "separable"), ("fp32", 33, 20, 0.6, "separable"),
    ("fp64", 24, 37, 0.3, "sum"), ("fp32", 40, 70, 0.0, "sum")])
def test_separable_coefficients(oracle_lib, precision, nk, nw, beta, envelope):
    pow2 = lambda n: 1 << max(1, (2 * n - 1).bit_length())  # noqa: E731
    wl = dataclasses.replace(sep_case(nk=nk, nw=nw, nx=pow2(nk), nt=pow2(nw),
                                      precision=precision, envelope=envelope), beta=beta)
    op = oracle_plan(wl)
    seeds = [3, 11, 2 ** 40 + 1]
    with srm3.Plan.create(wl, eps=op.eps) as p:
        C = _cplx(p.coeffs(seeds))
    # FP32: a radix-2 FFT convolution's rounding is bounded by about
    # log2(Nk Nw) u sum |z|^2 (u = 2^-24) for every output at once, 14 x 6e-8 x
    # the norm of z on these grids, so the bound is taken as 1e-5 of max|C|
    # (the O(N^2) kernel holds 2e-6); the fields stay within 1e-4 sigma_u below
    tol = 1e-11 if precision == "fp64" else 1e-5
    for i, s in enumerate(seeds):
        ref = op.coeffs(s)
        scale = np.abs(ref).max()
        assert np.abs(C[i] - ref).max() <= tol * scale


@pytest.mark.parametrize("precision,envelope", [("fp64", "separable"), ("fp32", "separable"),
                                                ("fp32", "sum")])
def test_separable_field_end_to_end(oracle_lib, precision, envelope):
    wl = sep_case(precision=precision, seeds=(1, 7), envelope=envelope)
    op = oracle_plan(wl)
    sig = math.sqrt(op.moments()[0])
    with srm3.Plan.create(wl) as p:
        u = p.sample(list(wl.seeds)).cpu().numpy()
    ref = np.stack([op.field(s, wl.n_x, wl.n_t) for s in wl.seeds])
    tol = 1e-10 if precision == "fp64" else 1e-4
    assert np.abs(u - ref).max() <= tol * sig


def test_separable_in_a_batch_is_bit_identical_to_alone():
    """A batch holding a separable plan next to Gaussian ones (one of them
    with a stored W table) gives each plan the fields of srm3_sample."""
    sep = sep_case(precision="fp32", seeds=(5, 6, 7))
    g1 = W.small_case(nk=24, nw=37, precision="fp32", storage="recompute", seeds=(1, 2))
    g2 = W.small_case(nk=16, nw=20, nx=32, nt=64, precision="fp32", storage="table",
                      seeds=(9,))
    wls = [sep, g1, g2]
    plans = [srm3.Plan.create(w) for w in wls]
    try:
        alone = [p.sample(list(w.seeds)).clone() for p, w in zip(plans, wls)]
        outs = [torch.empty_like(a) for a in alone]
        seeds = [s for w in wls for s in w.seeds]
        with srm3.Batch(plans, [w.n_samples for w in wls], outs) as b:
            b.run(seeds)
            b.sync()
        torch.cuda.synchronize()
        for a, o in zip(alone, outs):
            assert torch.equal(a, o)
    finally:
        for p in plans:
            p.destroy()


@pytest.mark.parametrize("envelope,precision,beta", [("gauss", "fp64", 0.0), ("gauss", "fp32", 0.4),
                                                     ("separable", "fp64", 0.3),
                                                     ("sum", "fp64", -0.5)])
def test_exact_moments_against_oracle(oracle_lib, envelope, precision, beta):
    """srm3_plan_moments: the exact variance and third moment against the
    oracle's direct sums over (S_p, b_p) at the same eps."""
    wl = dataclasses.replace(W.small_case(nk=24, nw=37, precision=precision), beta=beta,
                             envelope=envelope)
    S = oracle.kaimal_lorentzian(wl.n_kappa, wl.n_omega, wl.kappa_u, wl.omega_u, wl.U, wl.z,
                                 wl.z0, wl.k_vk, wl.lam)
    if envelope == "gauss":
        env = oracle.Envelope("gauss", wl.sigma_g)
    else:
        a, b = wl.envelope_tables()
        env = oracle.Envelope("separable", table=a, table_b=b)
    with srm3.Plan.create(wl) as p:
        eps = p.info().eps
        var, m3 = p.moments()
    op = oracle.make_plan(S, wl.kappa_u, wl.omega_u, eps=eps, env=env, beta=beta)
    ovar, om3 = op.moments()
    assert var == pytest.approx(ovar, rel=1e-12)
    assert abs(om3) > 1e-3 * ovar ** 1.5
    assert m3 == pytest.approx(om3, rel=1e-11)
