"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 plans max|du| <= 1e-10 sigma_u, FP32 plans max|du| <=
1e-4 sigma_u (sigma_u^2 = the exact ensemble variance); Philox words
bit-exact; plan tables (FP64 in both precisions) to 1e-11 relative.
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


@functools.lru_cache(maxsize=None)
def oracle_plan(wl, eps=None):
    S = oracle.kaimal_lorentzian(wl.n_kappa, wl.n_omega, wl.kappa_u, wl.omega_u, wl.U, wl.z,
                                 wl.z0, wl.k_vk, wl.lam)
    env = oracle.Envelope("gauss", wl.sigma_g)
    if eps is None:
        return oracle.make_plan(S, wl.kappa_u, wl.omega_u, target=wl.target, env=env,
                                beta=wl.beta)
    return oracle.make_plan(S, wl.kappa_u, wl.omega_u, eps=eps, env=env, beta=wl.beta)


def sigma_u(op):
    return math.sqrt(op.moments()[0])


def oracle_fields(op, wl, seeds):
    return np.stack([op.field(s, wl.n_x, wl.n_t) for s in seeds])


SMALL = W.small_case(nk=24, nw=37, nx=64, nt=128, seeds=(1, 2, 3, 77))


def test_phase_words_bit_exact(oracle_lib):
    wl = SMALL
    seeds = [1, 2, 2 ** 40 + 5, 2 ** 64 - 1]
    with srm3.Plan.create(wl) as p:
        w = p.phase_words(seeds).cpu().numpy().view(np.uint32)
    for i, s in enumerate(seeds):
        ref, _ = oracle.phases(wl.n_kappa, wl.n_omega, s)
        np.testing.assert_array_equal(w[i], ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_plan_tables_and_eps(oracle_lib, precision):
    wl = SMALL
    op = oracle_plan(wl)
    with srm3.Plan.create(wl, precision=precision) as p:
        S, q, sb2 = p.tables()
        info = p.info()
    # FP64 plans meet the target to 1e-13 (as the oracle's bisection);
    # FP32 plans to 1e-9, which moves eps and q by ~1e-9 relative
    tol, rel = (1e-13, 1e-11) if precision == "fp64" else (1e-9, 2e-8)
    np.testing.assert_allclose(S, op.S, rtol=1e-13, atol=0)
    assert info.eps == pytest.approx(op.eps, rel=rel)
    assert abs(info.max_sum_b2 - wl.target) <= tol
    np.testing.assert_allclose(q, op.q, rtol=rel)
    np.testing.assert_allclose(sb2, op.sum_b2, rtol=rel, atol=1e-15)
    assert info.variance == pytest.approx(op.moments()[0], rel=1e-12)
    assert np.all(q >= 1.0) and info.min_pure_ratio > 0
    # the Gaussian envelope (sigma_g = 0.25) runs the recursion in separable
    # form; FP32 plans take one FP64 pass and the first-order move of the
    # tables to the root, FP64 plans one FP64 pass at three values of eps^2
    # around the FP32 root and the tables interpolated to the root
    assert info.recursion_flags & srm3.SRM3_REC_SEPARABLE
    moved = bool(info.recursion_flags & srm3.SRM3_REC_TABLES_MOVED)
    interp = bool(info.recursion_flags & srm3.SRM3_REC_TABLES_INTERPOLATED)
    assert moved == (precision == "fp32") and interp == (precision == "fp64")
    assert info.root_passes == 1


@pytest.mark.parametrize("sigma_g,separable", [(0.15, False), (0.35, True)])
def test_recursion_envelope_width(oracle_lib, sigma_g, separable):
    """The Gaussian envelope splits as a^2_i a^2_j b^2_k on the pairs of a
    point; the recursion uses the split while the factors' exponent range
    ((Nk-1)/(sg Nk))^2 + ((Nw-1)/(sg Nw))^2 stays within 40, else the g^2
    table.  Both forms against the oracle's g^2 at a common eps, through
    several bulk phases and fringe blocks, and the eps search of an FP32
    plan with its tables moved to the root."""
    import dataclasses
    wl = dataclasses.replace(W.small_case(nk=48, nw=72, nx=64, nt=256), sigma_g=sigma_g)
    op = oracle_plan(wl)
    with srm3.Plan.create(wl, eps=op.eps, precision="fp64") as p:
        _, q, sb2 = p.tables()
        assert bool(p.info().recursion_flags & srm3.SRM3_REC_SEPARABLE) == separable
    np.testing.assert_allclose(q, op.q, rtol=2e-14)
    np.testing.assert_allclose(sb2, op.sum_b2, rtol=2e-14, atol=1e-16)
    # the eps search of an FP64 plan: tables interpolated from the three-plane
    # FP64 pass, in either form of the recursion
    with srm3.Plan.create(wl, precision="fp64") as p:
        _, q, sb2 = p.tables()
        info = p.info()
    assert info.recursion_flags & srm3.SRM3_REC_TABLES_INTERPOLATED
    assert info.eps == pytest.approx(op.eps, rel=1e-11)
    assert abs(info.max_sum_b2 - wl.target) <= 1e-13
    np.testing.assert_allclose(q, op.q, rtol=1e-11)
    np.testing.assert_allclose(sb2, op.sum_b2, rtol=1e-11, atol=1e-16)
    with srm3.Plan.create(wl, precision="fp32") as p:
        _, q, sb2 = p.tables()
        info = p.info()
    assert info.eps == pytest.approx(op.eps, rel=2e-8)
    assert abs(info.max_sum_b2 - wl.target) <= 1e-9
    np.testing.assert_allclose(q, op.q, rtol=2e-8)
    np.testing.assert_allclose(sb2, op.sum_b2, rtol=2e-8, atol=1e-15)


@pytest.mark.parametrize("mask", ["full", "no_coarse_pairs", "window_missed"])
def test_eps_search_coarse_start(mask):
    """The eps search of a 256 x 256 lattice starts from the root on the
    64 x 64 lattice of every fourth point per axis.  Since b_p^2 = x dk dw g^2
    q_i q_j, sum_b2 depends on S only through its support, so supports that
    the coarse lattice misreads steer the search down its fallbacks: S = 0 on
    the columns kw = 0 mod 4 leaves the coarse lattice without pairs, S = 0
    on kw = 2 mod 4 puts its root far from this lattice's (outside the
    bracketing pass's window).  Each way the FP32 plan meets the target to
    1e-9 and its eps agrees with the FP64 plan's (target to 1e-13, FP64
    passes to the end) to 2e-8."""
    wl = W.small_case(nk=256, nw=256, nx=256, nt=512, seeds=(1,))
    S = oracle.kaimal_lorentzian(256, 256, wl.kappa_u, wl.omega_u, wl.U, wl.z, wl.z0,
                                 wl.k_vk, wl.lam)
    if mask == "no_coarse_pairs":
        S[:, 0::4] = 0.0
    elif mask == "window_missed":
        S[:, 2::4] = 0.0
    res = {}
    for precision in ("fp64", "fp32"):
        with srm3.Plan.create(wl, table=S, precision=precision) as p:
            res[precision] = p.info()
    i32, i64 = res["fp32"], res["fp64"]
    for info in (i32, i64):
        assert (info.coarse_fk, info.coarse_fw) == (4, 4)
        started = bool(info.recursion_flags & srm3.SRM3_REC_COARSE_START)
        assert started == (mask == "full")
    assert abs(i64.max_sum_b2 - wl.target) <= 1e-13
    assert abs(i32.max_sum_b2 - wl.target) <= 1e-9
    assert i32.eps == pytest.approx(i64.eps, rel=2e-8)
    if mask == "no_coarse_pairs":
        assert i32.coarse_passes == 0  # the coarse linear bound found no pairs


@pytest.mark.parametrize("nk,nw,fk,fw", [(300, 260, 4, 4), (1100, 60, 16, 1)])
def test_eps_search_coarse_start_ragged(nk, nw, fk, fw):
    """Lattices that the coarse factors do not divide (the coarse lattice takes
    points 0, fk, 2 fk, ... below n_kappa), and one coarsened along kappa
    alone: the FP32 plan meets the target to 1e-9 and agrees with the FP64
    plan to 2e-8."""
    pow2 = lambda n: 1 << max(1, (2 * n - 1).bit_length())  # noqa: E731
    wl = W.small_case(nk=nk, nw=nw, nx=pow2(nk), nt=pow2(nw), seeds=(1,))
    res = {}
    for precision in ("fp64", "fp32"):
        with srm3.Plan.create(wl, precision=precision) as p:
            res[precision] = p.info()
    for info in res.values():
        assert (info.coarse_fk, info.coarse_fw) == (fk, fw)
    assert abs(res["fp64"].max_sum_b2 - wl.target) <= 1e-13
    assert abs(res["fp32"].max_sum_b2 - wl.target) <= 1e-9
    assert res["fp32"].eps == pytest.approx(res["fp64"].eps, rel=2e-8)


@pytest.mark.parametrize("nk,nw", [(40, 33), (96, 64), (130, 20), (12, 200)])
def test_recursion_at_fixed_eps(oracle_lib, nk, nw):
    """Same eps on both sides: the anti-diagonal recursion equals the
    lexicographic one to FP64 rounding.  The shapes take the pass through
    several bulk phases and fringe blocks, points with more than 32 row
    pairs (96 x 64, 130 x 20) and rows far longer than the lattice is tall."""
    pow2 = lambda n: 1 << max(1, (2 * n - 1).bit_length())  # noqa: E731
    wl = W.small_case(nk=nk, nw=nw, nx=pow2(nk), nt=pow2(nw))
    op = oracle_plan(wl)
    with srm3.Plan.create(wl, eps=op.eps, precision="fp64") as p:
        _, q, sb2 = p.tables()
    np.testing.assert_allclose(q, op.q, rtol=2e-14)
    np.testing.assert_allclose(sb2, op.sum_b2, rtol=2e-14, atol=1e-16)


def _cplx(C):
    C = C.cpu().numpy()
    return C[..., 0] + 1j * C[..., 1]


@pytest.mark.parametrize("precision,storage", [("fp64", "recompute"), ("fp32", "recompute"),
                                               ("fp32", "table")])
def test_coefficients(oracle_lib, precision, storage):
    wl = SMALL
    op = oracle_plan(wl)
    seeds = [3, 11]
    with srm3.Plan.create(wl, precision=precision, storage=storage, eps=op.eps) as p:
        C = _cplx(p.coeffs(seeds))
        info = p.info()
        assert info.storage == {"recompute": 2, "table": 1}[storage]
        # W recomputed for the Gaussian envelope: the FP32 pair sum multiplies
        # phasor rows scaled by the envelope's separable factors
        sepf = bool(info.recursion_flags & srm3.SRM3_PAIRSUM_SEPARABLE)
        assert sepf == (precision == "fp32" and storage == "recompute")
    tol = 1e-11 if precision == "fp64" else 2e-6
    for i, s in enumerate(seeds):
        ref = op.coeffs(s)
        scale = np.abs(ref).max()
        assert np.abs(C[i] - ref).max() <= tol * scale


def test_field_tiny_fp64_end_to_end(oracle_lib):
    """The 32 x 32 FP64 plain-method case: spectrum, eps search, phases,
    pair sum and transform on the GPU vs the oracle's own bisection."""
    wl = W.TINY
    op = oracle_plan(wl)
    with srm3.Plan.create(wl) as p:
        u = p.sample(list(wl.seeds)).cpu().numpy()
    ref = oracle_fields(op, wl, wl.seeds)
    err = np.abs(u - ref).max() / sigma_u(op)
    assert err <= 1e-10, err


@pytest.mark.parametrize("storage", ["recompute", "table"])
def test_field_small_fp32_end_to_end(oracle_lib, storage):
    wl = SMALL
    op = oracle_plan(wl)
    with srm3.Plan.create(wl, storage=storage) as p:
        u = p.sample(list(wl.seeds)).cpu().numpy()
    ref = oracle_fields(op, wl, wl.seeds)
    err = np.abs(u - ref).max() / sigma_u(op)
    assert err <= 1e-4, err


@pytest.mark.parametrize("nk,nw,nx,nt", [(1, 9, 2, 32), (2, 3, 2, 8), (9, 1, 16, 2),
                                         (17, 16, 32, 32), (8, 64, 8, 128)])
def test_edge_lattices_fp64(oracle_lib, nk, nw, nx, nt):
    """One-row and one-column lattices (N_kappa = 1 is the 1-D form),
    minimal sizes, n_x = n_kappa and n_t = 2 n_omega - 1 rounded up."""
    wl = W.small_case(nk=nk, nw=nw, nx=nx, nt=nt, seeds=(4, 5), precision="fp64")
    S = oracle.kaimal_lorentzian(nk, nw, wl.kappa_u, wl.omega_u, wl.U, wl.z)
    eps = 0.2
    op = oracle.make_plan(S, wl.kappa_u, wl.omega_u, eps=eps, env=oracle.Envelope("gauss", 0.25))
    with srm3.Plan.create(wl, eps=eps) as p:
        u = p.sample(list(wl.seeds)).cpu().numpy()
    ref = oracle_fields(op, wl, wl.seeds)
    sig = max(sigma_u(op), 1e-300)
    assert np.abs(u - ref).max() <= 1e-10 * sig + 1e-300


def test_eps_zero_and_biphase(oracle_lib):
    wl = W.small_case(nk=12, nw=10, nx=16, nt=32, seeds=(9,), beta=0.7, precision="fp64")
    for eps in (0.0, 0.9):
        S = oracle.kaimal_lorentzian(12, 10, wl.kappa_u, wl.omega_u, wl.U, wl.z)
        op = oracle.make_plan(S, wl.kappa_u, wl.omega_u, eps=eps,
                              env=oracle.Envelope("gauss", 0.25), beta=0.7)
        with srm3.Plan.create(wl, eps=eps) as p:
            u = p.sample([9]).cpu().numpy()[0]
        ref = op.field(9, wl.n_x, wl.n_t)
        assert np.abs(u - ref).max() <= 1e-10 * sigma_u(op)


def test_spectrum_table_input(oracle_lib):
    rng = np.random.default_rng(1)
    wl = W.small_case(nk=10, nw=12, nx=16, nt=32, seeds=(2,), precision="fp64")
    S = rng.uniform(0.0, 3.0, size=(10, 12))
    S[0, 0] = 1.5          # a positive DC entry takes part in no pair
    S[3, 4] = 0.0
    op = oracle.make_plan(S, wl.kappa_u, wl.omega_u, target=0.4,
                          env=oracle.Envelope("gauss", 0.25))
    with srm3.Plan.create(wl, table=S, target=0.4) as p:
        u = p.sample([2]).cpu().numpy()[0]
        _, q, _ = p.tables()
    np.testing.assert_allclose(q, op.q, rtol=1e-11)
    ref = op.field(2, wl.n_x, wl.n_t)
    assert np.abs(u - ref).max() <= 1e-10 * sigma_u(op)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_transform_alone(oracle_lib, precision):
    rng = np.random.default_rng(3)
    wl = W.small_case(nk=20, nw=24, nx=32, nt=64, precision=precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    Cn = rng.normal(size=(3, 2, 20, 24)) + 1j * rng.normal(size=(3, 2, 20, 24))
    C = torch.tensor(np.stack([Cn.real, Cn.imag], -1), dtype=dt, device="cuda")
    with srm3.Plan.create(wl, eps=0.0) as p:
        u = p.field_from_coeffs(C).cpu().numpy()
    tol = 1e-12 if precision == "fp64" else 2e-6
    for i in range(3):
        ref = oracle.field_dft(Cn[i], 32, 64)
        assert np.abs(u[i] - ref).max() <= tol * np.abs(ref).max()
        # cuFFT cross-check (library, not the oracle)
        F = torch.zeros((32, 64), dtype=torch.complex128, device="cuda")
        Ct = torch.tensor(Cn[i], device="cuda")
        F[:20, :24] += Ct[0]
        idx = (-torch.arange(24, device="cuda")) % 64
        F[:20].index_add_(1, idx, Ct[1])
        cu = (torch.fft.ifft2(F) * (32 * 64)).real.cpu().numpy()
        assert np.abs(u[i] - cu).max() <= tol * np.abs(cu).max()


# (nk, nw, nx, nt): lattices that leave most inputs of a stage's first pass
# zero, so that the FP32 transform takes its pruned first passes -- x stage
# with 1, 4, 4 nonzero blocks at each end, t stage with 2, 1, 2 (blocks of
# L/R inputs, R = 16 the first radix at these lengths)
PRUNED_CASES = [(8, 16, 128, 256), (30, 7, 128, 256), (40, 20, 256, 512)]


@pytest.mark.parametrize("nk,nw,nx,nt", PRUNED_CASES)
def test_transform_pruned_first_passes(oracle_lib, nk, nw, nx, nt):
    """The first pass of each transform stage skips the butterflies of inputs
    that are zero by construction (coefficients only at kk < nk or nx - kk
    < nk, and the t rows only at m < nw or nt/2 - m < nw): against the
    oracle's direct double sum and cuFFT, 2e-6 of max|u|."""
    rng = np.random.default_rng(nk * 1000 + nw)
    wl = W.small_case(nk=nk, nw=nw, nx=nx, nt=nt, precision="fp32")
    Cn = rng.normal(size=(2, 2, nk, nw)) + 1j * rng.normal(size=(2, 2, nk, nw))
    C = torch.tensor(np.stack([Cn.real, Cn.imag], -1), dtype=torch.float32, device="cuda")
    with srm3.Plan.create(wl, eps=0.0) as p:
        u = p.field_from_coeffs(C).cpu().numpy()
    for i in range(2):
        ref = oracle.field_dft(Cn[i], nx, nt)
        assert np.abs(u[i] - ref).max() <= 2e-6 * np.abs(ref).max()
        F = torch.zeros((nx, nt), dtype=torch.complex128, device="cuda")
        Ct = torch.tensor(Cn[i], device="cuda")
        F[:nk, :nw] += Ct[0]
        idx = (-torch.arange(nw, device="cuda")) % nt
        F[:nk].index_add_(1, idx, Ct[1])
        cu = (torch.fft.ifft2(F) * (nx * nt)).real.cpu().numpy()
        assert np.abs(u[i] - cu).max() <= 2e-6 * np.abs(cu).max()


def test_batch_composition_and_chunking(oracle_lib):
    """A seed's field is bit-identical alone, inside a batch, and across the
    internal 128-sample chunk boundary."""
    wl = W.small_case(nk=16, nw=20, nx=16, nt=64)
    with srm3.Plan.create(wl) as p:
        alone = p.sample([5]).cpu().numpy()[0]
        mix = p.sample(list(range(1, 10))).cpu().numpy()
        big = p.sample(list(range(1000, 1131))).cpu().numpy()
        tail = p.sample([1130]).cpu().numpy()[0]
        head = p.sample([1000]).cpu().numpy()[0]
        assert p.sample([]).numel() == 0
    np.testing.assert_array_equal(mix[4], alone)
    np.testing.assert_array_equal(big[130], tail)
    np.testing.assert_array_equal(big[0], head)


def test_nonpositive_pure_is_reported(oracle_lib):
    wl = W.small_case(nk=12, nw=12)
    with pytest.raises(srm3.SRM3Error) as ei:
        srm3.Plan.create(wl, eps=50.0)
    assert ei.value.code == -3


def test_sample_host_matches_device(oracle_lib):
    wl = W.small_case(nk=16, nw=20, nx=16, nt=64)
    with srm3.Plan.create(wl) as p:
        dev = p.sample([7, 8]).cpu().numpy()
        host = torch.empty((2, 16, 64), dtype=torch.float32).pin_memory()
        srm3.sample_host(p.handle, [7, 8], 2, host.data_ptr())
    np.testing.assert_array_equal(host.numpy(), dev)
