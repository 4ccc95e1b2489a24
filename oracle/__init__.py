"""FP64 CPU oracle for the third-order SRM stochastic wave (arXiv 2310.03979).

Test infrastructure only: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The oracle shares no code
with the CUDA library and imports nothing from it; the arithmetic lives in
``srm3_oracle.c`` (plain C, FP64, OpenMP over independent outputs) and this
module only marshals numpy arrays through ctypes.

Parity status per function (what pins it, see ``tests/test_oracle_pins.py``):
  kaimal_lorentzian  closed form of the Kaimal spectrum and the Lorentzian's
                     unit integral (Sec. 5, Eqs. kaimal_spectrum and
                     kaimal_davenport_spectrum)
  recursion          hand-worked 3x3 lattice, separable-envelope FFT
                     self-convolution, scale invariance (Eq. pure)
  recursion_mixed    the plain recursion when no difference pair carries
                     weight; a hand-worked 2x4 lattice with difference pairs;
                     the fixed-point residual; scale invariance
  bisect_eps         monotonicity and the target it reaches
  philox4x32_10      cuRAND's host Philox4_32_10 generator (library)
  phases             counter/key map of the same generator
  coeffs             ordered-pair brute force, separable FFT convolution,
                     eps = 0 reduction to the 2nd-order SRM (Sec. 3); with
                     difference pairs, a brute force over all ordered pairs
                     of signed lattice points
  field_dft          numpy FFT of the same coefficients
  field_series       equals coefficients + DFT (FFT form, Sec. 4.3)
  exact_moments      Monte Carlo moments of the series over many seeds;
                     with difference pairs, the closed form in S and g
                     alone and a Monte Carlo skewness
  field_stats        closed-form moments of a sampled sinusoid, a centred
                     uniform grid and a two-point distribution; exact bin
                     counts of the uniform grid (sample statistics, Sec. 6)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "srm3_oracle.c")
_LIB = os.path.join(_HERE, "libsrm3_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile ``srm3_oracle.c`` into ``libsrm3_oracle.so`` (OpenMP if gcc has it)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
            _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i, d, u64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64
        lib.or_kaimal_lorentzian.argtypes = [i, i, d, d, d, d, d, d, d, dp]
        lib.or_recursion.argtypes = [i, i, d, d, dp, i, d, dp, d, dp, dp]
        lib.or_recursion_mixed.argtypes = [i, i, d, d, dp, i, d, dp, d, d, i, dp, dp, ip]
        lib.or_bisect_eps.argtypes = [i, i, d, d, dp, i, d, dp, i, d, d, i, dp, dp,
                                      ip, dp, dp]
        lib.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.or_philox4x32_10.restype = None
        lib.or_phases.argtypes = [i, i, u64, u32p, dp]
        lib.or_phases.restype = None
        lib.or_coeffs.argtypes = [i, i, d, d, dp, dp, i, d, dp, i, d, d, u64, dp]
        lib.or_field_dft.argtypes = [i, i, i, i, dp, dp]
        lib.or_field_points.argtypes = [i, i, i, i, dp, i, ip, ip, dp]
        lib.or_field_series.argtypes = [i, i, d, d, i, i, dp, dp, i, d, dp, i, d, d,
                                        u64, i, ip, ip, dp]
        lib.or_exact_moments.argtypes = [i, i, d, d, dp, dp, i, d, dp, i, d, d, dp, dp]
        lib.or_num_threads.argtypes = []
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


@dataclass
class Envelope:
    """Bispectrum envelope g(i, j): ``kind='gauss'`` with width ``sigma_g``
    (fraction of the lattice extent per axis), or ``kind='separable'`` with
    g = e(i) e(j) e(i+j) from ``table`` of shape (Nk, Nw), or, when
    ``table_b`` is given too, g = a(i) a(j) b(i+j) with a = ``table`` and
    b = ``table_b``."""
    kind: str = "gauss"
    sigma_g: float = 0.25
    table: np.ndarray | None = None
    table_b: np.ndarray | None = None

    def args(self, nk, nw):
        if self.kind == "gauss":
            return 0, float(self.sigma_g), None
        if self.kind == "separable":
            t = np.ascontiguousarray(self.table, dtype=np.float64)
            assert t.shape == (nk, nw)
            if self.table_b is None:
                return 1, 0.0, t
            b = np.ascontiguousarray(self.table_b, dtype=np.float64)
            assert b.shape == (nk, nw)
            return 2, 0.0, np.ascontiguousarray(np.concatenate([t.ravel(), b.ravel()]))
        raise ValueError(self.kind)


def _env(env, nk, nw):
    kind, sg, tab = (env or Envelope()).args(nk, nw)
    return kind, sg, tab, (_dp(tab) if tab is not None else None)


def num_threads() -> int:
    return int(_load().or_num_threads())


def kaimal_lorentzian(nk, nw, kappa_u, omega_u, U, z, z0=0.03, k_vk=0.4, lam=7.0):
    """S(kappa_k, omega_k) on the lattice, shape (Nk, Nw) (Sec. 5)."""
    S = np.zeros((nk, nw), dtype=np.float64)
    _check(_load().or_kaimal_lorentzian(nk, nw, kappa_u, omega_u, U, z, z0, k_vk,
                                        lam, _dp(S)), "kaimal_lorentzian")
    return S


def recursion(S, kappa_u, omega_u, eps, env=None):
    """Pure spectrum S_p and sum_b2 at a given eps (Eq. pure), lexicographic order."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    nk, nw = S.shape
    kind, sg, tab, tabp = _env(env, nk, nw)
    Sp = np.zeros_like(S)
    sb2 = np.zeros_like(S)
    _check(_load().or_recursion(nk, nw, kappa_u, omega_u, _dp(S), kind, sg, tabp,
                                eps, _dp(Sp), _dp(sb2)), "recursion")
    return Sp, sb2


def recursion_mixed(S, kappa_u, omega_u, eps, env=None, tol=1e-15, max_sweeps=100000):
    """Pure spectrum with sum and difference (mixed-sign) interactions: the
    largest fixed point of Eq. pure by lexicographic Gauss-Seidel sweeps from
    S_p = S.  Returns (S_p, sum_b2, sweeps)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    nk, nw = S.shape
    kind, sg, tab, tabp = _env(env, nk, nw)
    Sp = np.zeros_like(S)
    sb2 = np.zeros_like(S)
    sw = ctypes.c_int()
    _check(_load().or_recursion_mixed(nk, nw, kappa_u, omega_u, _dp(S), kind, sg, tabp,
                                      eps, tol, max_sweeps, _dp(Sp), _dp(sb2),
                                      ctypes.byref(sw)), "recursion_mixed")
    return Sp, sb2, sw.value


def bisect_eps(S, kappa_u, omega_u, target, env=None, tol=1e-13, max_iter=200,
               mixed=False):
    """FP64 bisection on eps so that max_k sum_b2 = target (with difference
    interactions when ``mixed``).
    Returns (eps, max_sum_b2, evaluations, S_p, sum_b2)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    nk, nw = S.shape
    kind, sg, tab, tabp = _env(env, nk, nw)
    Sp = np.zeros_like(S)
    sb2 = np.zeros_like(S)
    eps = ctypes.c_double()
    mx = ctypes.c_double()
    it = ctypes.c_int()
    _check(_load().or_bisect_eps(nk, nw, kappa_u, omega_u, _dp(S), kind, sg, tabp,
                                 int(bool(mixed)), target, tol, max_iter, ctypes.byref(eps),
                                 ctypes.byref(mx), ctypes.byref(it), _dp(Sp),
                                 _dp(sb2)), "bisect_eps")
    return eps.value, mx.value, it.value, Sp, sb2


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_u32p(c), _u32p(k), _u32p(out))
    return out


def phases(nk, nw, seed):
    """(words, phi), each shape (2, Nk, Nw): sheet 0 = +omega, sheet 1 = -omega."""
    words = np.zeros((2, nk, nw), dtype=np.uint32)
    phi = np.zeros((2, nk, nw), dtype=np.float64)
    _load().or_phases(nk, nw, int(seed), _u32p(words), _dp(phi))
    return words, phi


def coeffs(S, Sp, kappa_u, omega_u, eps, seed, env=None, beta=0.0, mixed=False):
    """C^s_k, complex128 shape (2, Nk, Nw) (FFT form, Sec. 4.3); ``mixed``
    adds the difference pairs."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    Sp = np.ascontiguousarray(Sp, dtype=np.float64)
    nk, nw = S.shape
    kind, sg, tab, tabp = _env(env, nk, nw)
    C = np.zeros((2, nk, nw, 2), dtype=np.float64)
    _check(_load().or_coeffs(nk, nw, kappa_u, omega_u, _dp(S), _dp(Sp), kind, sg,
                             tabp, int(bool(mixed)), eps, beta, int(seed), _dp(C)),
           "coeffs")
    return C[..., 0] + 1j * C[..., 1]


def _cpack(C):
    C = np.asarray(C, dtype=np.complex128)
    out = np.empty(C.shape + (2,), dtype=np.float64)
    out[..., 0] = C.real
    out[..., 1] = C.imag
    return np.ascontiguousarray(out)


def field_dft(C, nx, nt):
    """u[mx, mt] from coefficients by the direct (separable) double sum."""
    Cp = _cpack(C)
    _, nk, nw, _ = Cp.shape
    u = np.zeros((nx, nt), dtype=np.float64)
    _check(_load().or_field_dft(nk, nw, nx, nt, _dp(Cp), _dp(u)), "field_dft")
    return u


def field_points(C, nx, nt, mx, mt):
    """u at points (mx[p], mt[p]) by the plain double sum over all coefficients."""
    Cp = _cpack(C)
    _, nk, nw, _ = Cp.shape
    mx = np.ascontiguousarray(mx, dtype=np.int32)
    mt = np.ascontiguousarray(mt, dtype=np.int32)
    u = np.zeros(len(mx), dtype=np.float64)
    _check(_load().or_field_points(nk, nw, nx, nt, _dp(Cp), len(mx), _ip(mx),
                                   _ip(mt), _dp(u)), "field_points")
    return u


def field_series(S, Sp, kappa_u, omega_u, eps, seed, nx, nt, mx, mt, env=None,
                 beta=0.0, mixed=False):
    """u at points by the literal cosine series (Eq. quadrant_1d_wave; its
    mixed cosines too when ``mixed``)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    Sp = np.ascontiguousarray(Sp, dtype=np.float64)
    nk, nw = S.shape
    kind, sg, tab, tabp = _env(env, nk, nw)
    mx = np.ascontiguousarray(mx, dtype=np.int32)
    mt = np.ascontiguousarray(mt, dtype=np.int32)
    u = np.zeros(len(mx), dtype=np.float64)
    _check(_load().or_field_series(nk, nw, kappa_u, omega_u, nx, nt, _dp(S), _dp(Sp),
                                   kind, sg, tabp, int(bool(mixed)), eps, beta,
                                   int(seed), len(mx),
                                   _ip(mx), _ip(mt), _dp(u)), "field_series")
    return u


def exact_moments(S, Sp, kappa_u, omega_u, eps, env=None, beta=0.0, mixed=False):
    """(variance, third moment) of the discrete series over the phases."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    Sp = np.ascontiguousarray(Sp, dtype=np.float64)
    nk, nw = S.shape
    kind, sg, tab, tabp = _env(env, nk, nw)
    v = ctypes.c_double()
    m3 = ctypes.c_double()
    _check(_load().or_exact_moments(nk, nw, kappa_u, omega_u, _dp(S), _dp(Sp), kind,
                                    sg, tabp, int(bool(mixed)), eps, beta, ctypes.byref(v),
                                    ctypes.byref(m3)), "exact_moments")
    return v.value, m3.value


@dataclass
class OraclePlan:
    """S, S_p and eps for one spectrum on one lattice."""
    S: np.ndarray
    Sp: np.ndarray
    sum_b2: np.ndarray
    eps: float
    kappa_u: float
    omega_u: float
    env: Envelope
    beta: float = 0.0
    mixed: bool = False

    @property
    def q(self):
        """q = S / S_p (1 where S = 0)."""
        out = np.ones_like(self.S)
        m = self.S > 0
        out[m] = self.S[m] / self.Sp[m]
        return out

    def coeffs(self, seed):
        return coeffs(self.S, self.Sp, self.kappa_u, self.omega_u, self.eps, seed,
                      self.env, self.beta, self.mixed)

    def field(self, seed, nx, nt):
        return field_dft(self.coeffs(seed), nx, nt)

    def moments(self):
        return exact_moments(self.S, self.Sp, self.kappa_u, self.omega_u, self.eps,
                             self.env, self.beta, self.mixed)


def make_plan(S, kappa_u, omega_u, *, target=None, eps=None, env=None, beta=0.0,
              tol=1e-13, mixed=False):
    """Oracle plan: eps from bisection on ``target`` (max sum_b2), or given;
    ``mixed`` adds the difference interactions."""
    env = env or Envelope()
    if target is not None:
        e, _, _, Sp, sb2 = bisect_eps(S, kappa_u, omega_u, target, env, tol=tol, mixed=mixed)
    else:
        e = float(eps)
        if mixed:
            Sp, sb2, _ = recursion_mixed(S, kappa_u, omega_u, e, env)
        else:
            Sp, sb2 = recursion(S, kappa_u, omega_u, e, env)
    return OraclePlan(np.ascontiguousarray(S, dtype=np.float64), Sp, sb2, e, kappa_u,
                      omega_u, env, beta, bool(mixed))


def field_stats(u, nbins, lo, hi, shift=0.0):
    """Sample statistics of field values (Sec. 6: sample mean, variance and
    skewness; empirical PDF and CDF by histogram), by their definitions.

    Power sums sum (u - shift)^p, p = 1..4, exactly rounded (math.fsum over
    FP64 terms; FP32 values convert exactly).  Bins: floor((u - lo) * scale)
    with scale = nbins / (hi - lo), both operations in the dtype of u and
    rounded once each (the precision the bin decision is taken in); below lo
    and at or above hi (or NaN) are counted apart.  Moments about the mean
    follow from the power sums."""
    import math
    u = np.asarray(u).ravel()
    dt = np.float32 if u.dtype == np.float32 else np.float64
    u = u.astype(dt, copy=False)
    d = u.astype(np.float64) - np.float64(shift)
    ps = [math.fsum((d ** p).tolist()) for p in (1, 2, 3, 4)]
    n = float(u.size)
    scale = dt(float(nbins) / (hi - lo))
    with np.errstate(invalid="ignore"):
        t = (u - dt(lo)) * scale
        below = int(np.count_nonzero(t < 0))
        inb = (t >= 0) & (t < nbins)
    above = int(u.size - below - np.count_nonzero(inb))
    hist = np.bincount(np.floor(t[inb]).astype(np.int64), minlength=nbins).astype(np.uint64)
    out = {"count": n, "power_sum": ps, "hist": hist, "below": below, "above": above}
    if n > 0:
        m1, e2, e3, e4 = (x / n for x in ps)
        c2 = e2 - m1 * m1
        c3 = e3 - 3 * m1 * e2 + 2 * m1 ** 3
        c4 = e4 - 4 * m1 * e3 + 6 * m1 * m1 * e2 - 3 * m1 ** 4
        out.update(mean=shift + m1, variance=c2,
                   skewness=c3 / c2 ** 1.5 if c2 > 0 else 0.0,
                   kurtosis=c4 / c2 ** 2 if c2 > 0 else 0.0)
    return out
