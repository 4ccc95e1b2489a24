"""Mixed-sign (difference) interactions on the GPU against the FP64 oracle.

The difference pairs (opposite-sign frequencies, Eq. truncated_cosines_1d_wave
and the mixed cosines of Eq. quadrant_1d_wave) make Eq. pure a fixed point.
The GPU iterates (difference sums at the previous iterate, then one level
pass in the Gauss-Seidel order of the plain recursion), the oracle sweeps
the lattice in lexicographic order; both converge from S_p = S to the same
largest fixed point, to a relative 4e-16 and 1e-15 per iteration.

Tolerances: plan tables at a common eps 1e-11 relative; FP64 plans meet the
target to 1e-13, FP32 plans to 1e-9 (q, eps within 2e-8); coefficients 1e-12
(FP64) and 2e-6 (FP32) of max|C|; fields 1e-10 sigma_u (FP64) and 1e-4
sigma_u (FP32), the tolerances of the plain model.
"""
import functools
import math

import numpy as np
import pytest

import oracle
from paper_2310_03979_gb300 import srm3
from paper_2310_03979_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _wl(nk, nw, nx=None, nt=None, seeds=(1, 2, 3), precision="fp32", beta=0.0,
        sigma_g=0.4, target=0.5):
    pow2 = lambda n: 1 << max(1, (n - 1).bit_length())  # noqa: E731
    c = W.small_case(nk=nk, nw=nw, nx=nx or pow2(nk), nt=nt or pow2(2 * nw - 1),
                     seeds=seeds, precision=precision, beta=beta, sigma_g=sigma_g,
                     target=target)
    from dataclasses import replace
    return replace(c, interactions="mixed")


@functools.lru_cache(maxsize=None)
def _oracle(wl, eps=None):
    S = oracle.kaimal_lorentzian(wl.n_kappa, wl.n_omega, wl.kappa_u, wl.omega_u, wl.U, wl.z,
                                 wl.z0, wl.k_vk, wl.lam)
    env = oracle.Envelope("gauss", wl.sigma_g)
    if eps is None:
        return oracle.make_plan(S, wl.kappa_u, wl.omega_u, target=wl.target, env=env,
                                beta=wl.beta, mixed=True)
    return oracle.make_plan(S, wl.kappa_u, wl.omega_u, eps=eps, env=env, beta=wl.beta,
                            mixed=True)


@pytest.mark.parametrize("nk,nw", [(24, 37), (40, 70), (1, 9), (9, 2), (33, 20)])
def test_mixed_tables_at_fixed_eps(oracle_lib, nk, nw):
    wl = _wl(nk, nw)
    eps = 0.3 if nk == 1 else 0.6  # the 1-D lattice has no fixed point at 0.6
    op = _oracle(wl, eps)
    with srm3.Plan.create(wl, precision="fp64", eps=eps) as p:
        S, q, sb2 = p.tables()
        info = p.info()
    assert info.interactions == srm3.SRM3_INTERACTIONS_MIXED
    assert info.fixed_point_iterations >= 2
    assert info.diff_pairs == wl.diff_pairs()
    np.testing.assert_allclose(q, op.q, rtol=1e-11)
    np.testing.assert_allclose(sb2, op.sum_b2, rtol=1e-11, atol=1e-16)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mixed_eps_search(oracle_lib, precision):
    wl = _wl(24, 37, precision=precision)
    op = _oracle(wl)
    with srm3.Plan.create(wl) as p:
        _, q, sb2 = p.tables()
        info = p.info()
    tol, rel = (1e-13, 1e-11) if precision == "fp64" else (1e-9, 2e-8)
    assert abs(info.max_sum_b2 - wl.target) <= tol
    assert info.eps == pytest.approx(op.eps, rel=rel)
    np.testing.assert_allclose(q, op.q, rtol=rel)
    # the difference pairs take part of the budget: a smaller eps than the plain model
    with srm3.Plan.create(wl, mixed=False) as p0:
        assert p0.info().eps > info.eps * 1.01


@pytest.mark.parametrize("precision,nk,nw,beta", [
    ("fp64", 24, 37, 0.0), ("fp32", 24, 37, 0.0), ("fp32", 40, 70, 0.6),
    ("fp64", 33, 20, 0.6), ("fp32", 1, 9, 0.0), ("fp32", 9, 2, 0.0), ("fp32", 130, 20, 0.0)])
def test_mixed_coefficients_and_fields(oracle_lib, precision, nk, nw, beta):
    wl = _wl(nk, nw, precision=precision, beta=beta, seeds=(1, 2, 77))
    eps = 0.3 if nk == 1 else 0.6
    op = _oracle(wl, eps)
    sig = math.sqrt(op.moments()[0])
    with srm3.Plan.create(wl, eps=eps) as p:
        C = p.coeffs(list(wl.seeds)).cpu().numpy()
        u = p.sample(list(wl.seeds)).cpu().numpy()
    C = C[..., 0] + 1j * C[..., 1]
    ctol, utol = (1e-12, 1e-10) if precision == "fp64" else (2e-6, 1e-4)
    for i, s in enumerate(wl.seeds):
        ref = op.coeffs(s)
        scale = np.abs(ref).max()
        assert np.abs(C[i] - ref).max() <= ctol * scale, (s, np.abs(C[i] - ref).max() / scale)
        uf = op.field(s, wl.n_x, wl.n_t)
        assert np.abs(u[i] - uf).max() <= utol * sig, (s, np.abs(u[i] - uf).max() / sig)


def test_mixed_fields_with_eps_search_and_positive_dc_column(oracle_lib):
    """A tabulated spectrum with S > 0 on the omega = 0 column (those points
    take sum pairs only) and holes, eps from the target, FP64 and FP32."""
    rng = np.random.default_rng(5)
    S = rng.uniform(0.2, 2.0, size=(12, 15))
    S[0, 0] = 0.0
    S[4, 6] = 0.0
    S[7, 0] = 0.0
    for precision, tol in (("fp64", 1e-10), ("fp32", 1e-4)):
        wl = _wl(12, 15, precision=precision, seeds=(3, 4), target=0.4)
        env = oracle.Envelope("gauss", wl.sigma_g)
        op = oracle.make_plan(S, wl.kappa_u, wl.omega_u, target=0.4, env=env, mixed=True)
        sig = math.sqrt(op.moments()[0])
        with srm3.Plan.create(wl, table=S, target=0.4) as p:
            u = p.sample(list(wl.seeds)).cpu().numpy()
        for i, s in enumerate(wl.seeds):
            err = np.abs(u[i] - op.field(s, wl.n_x, wl.n_t)).max() / sig
            assert err <= tol, (precision, s, err)


def test_mixed_exact_moments(oracle_lib):
    wl = _wl(20, 31, precision="fp64")
    op = _oracle(wl, 0.6)
    with srm3.Plan.create(wl, eps=0.6) as p:
        var, m3 = p.moments()
    v0, m30 = op.moments()
    assert var == pytest.approx(v0, rel=1e-12)
    assert m3 == pytest.approx(m30, rel=1e-11)


def test_mixed_bit_identical_alone_in_batch_and_across_counts():
    wl = _wl(24, 37, seeds=tuple(range(1, 41)))
    with srm3.Plan.create(wl, eps=0.6) as p:
        alone = p.sample([7])
        many = p.sample(list(range(1, 41)))  # full sample groups (half-group mode above)
        torch.cuda.synchronize()
        assert torch.equal(many[6], alone[0])
        other = W.small_case(nk=16, nw=20, nx=16, nt=64, seeds=(1, 2))
        with srm3.Plan.create(other) as q:
            outs = [torch.full((3, wl.n_x, wl.n_t), float("nan"), device="cuda"),
                    torch.full((2, 16, 64), float("nan"), device="cuda")]
            with srm3.Batch([p, q], [3, 2], outs) as b:
                b.run([5, 6, 7, 1, 2])
                b.sync()
            ref_p = p.sample([5, 6, 7])
            ref_q = q.sample([1, 2])
            torch.cuda.synchronize()
            assert torch.equal(outs[0], ref_p)
            assert torch.equal(outs[1], ref_q)


def test_mixed_rejects_table_storage_and_separable():
    wl = _wl(12, 12)
    with pytest.raises(srm3.SRM3Error) as ei:
        srm3.Plan.create(wl, storage="table", eps=0.5)
    assert ei.value.code == -8
    from dataclasses import replace
    sep = replace(W.BRIDGE_SEP, n_kappa=12, n_omega=12, n_x=16, n_t=32, interactions="mixed")
    with pytest.raises(srm3.SRM3Error) as ei:
        srm3.Plan.create(sep, eps=0.5)
    assert ei.value.code == -8
