"""ctypes binding of the SRM3 C ABI (``include/srm3.h``), same names as the C
calls.  Argument marshalling only: every step of the sampler runs in the CUDA
kernels of ``libsrm3.so``.  There is no CPU path; if the library cannot be
loaded (or built with nvcc), every call raises.

PyTorch is used only to hold device memory for the convenience wrappers
(``Plan.sample`` and friends); the raw calls take integer device pointers.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

SRM3_OK = 0
SRM3_ERR = {
    -1: "INVALID_ARG", -2: "GRID_CONSTRAINT", -3: "NONPOSITIVE_PURE",
    -4: "BISECTION_FAILED", -5: "OUT_OF_MEMORY", -6: "CUDA", -7: "TIMEOUT",
    -8: "NOT_SUPPORTED",
}
SRM3_SPECTRUM_KAIMAL_LORENTZIAN = 0
SRM3_SPECTRUM_TABLE = 1
SRM3_BISPECTRUM_GAUSS_ENVELOPE = 0
SRM3_BISPECTRUM_SEPARABLE = 1
SRM3_INTERACTIONS_SUM, SRM3_INTERACTIONS_MIXED = 0, 1
SRM3_FP32, SRM3_FP64 = 0, 1
SRM3_STORAGE_AUTO, SRM3_STORAGE_TABLE, SRM3_STORAGE_RECOMPUTE, SRM3_STORAGE_TUNED = 0, 1, 2, 3
EXPORTED = [
    "srm3_plan_create", "srm3_sample", "srm3_sample_host", "srm3_destroy", "srm3_sync",
    "srm3_set_stream", "srm3_last_error", "srm3_plan_info", "srm3_plan_tables",
    "srm3_plan_moments", "srm3_selftest_timeouts",
    "srm3_phase_words", "srm3_coeffs", "srm3_field_from_coeffs", "srm3_enable_timing",
    "srm3_get_timings", "srm3_field_from_coeffs_noalloc", "srm3_autotune",
    "srm3_batch_device_bytes", "srm3_set_tile_width",
    "srm3_batch_create", "srm3_batch_run", "srm3_batch_capture", "srm3_batch_sync",
    "srm3_batch_pair_terms", "srm3_batch_destroy", "srm3_batch_enable_timing",
    "srm3_batch_pairsum_ms", "srm3_batch_set_max_ctas",
    "srm3_stats_create", "srm3_stats_add", "srm3_stats_read", "srm3_stats_reset",
    "srm3_stats_destroy",
]
SRM3_STATS_MAX_BINS = 16384
SRM3_NOALLOC_SCRATCH_BYTES = 16 << 20


class srm3_tune_result(ctypes.Structure):
    _fields_ = [("table_ms", ctypes.c_double), ("recompute_ms", ctypes.c_double),
                ("storage", ctypes.c_int32), ("samples", ctypes.c_int32),
                ("tile_width", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("table_ms_w32", ctypes.c_double), ("table_ms_w16", ctypes.c_double),
                ("recompute_ms_w32", ctypes.c_double), ("recompute_ms_w16", ctypes.c_double)]


class srm3_spectrum(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("U", ctypes.c_double), ("z", ctypes.c_double), ("z0", ctypes.c_double),
                ("k_vk", ctypes.c_double), ("lam", ctypes.c_double),
                ("table", ctypes.POINTER(ctypes.c_double))]


class srm3_bispectrum(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("interactions", ctypes.c_int32),
                ("target_max_sum_b2", ctypes.c_double), ("eps", ctypes.c_double),
                ("sigma_g", ctypes.c_double), ("beta", ctypes.c_double),
                ("env_table", ctypes.POINTER(ctypes.c_double)),
                ("env_table_b", ctypes.POINTER(ctypes.c_double))]


class srm3_grid(ctypes.Structure):
    _fields_ = [("n_kappa", ctypes.c_int32), ("n_omega", ctypes.c_int32),
                ("kappa_u", ctypes.c_double), ("omega_u", ctypes.c_double),
                ("n_x", ctypes.c_int32), ("n_t", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("table_budget_bytes", ctypes.c_double),
                ("row_begin", ctypes.c_int32), ("row_end", ctypes.c_int32)]


# srm3_info.recursion_flags
SRM3_REC_SEPARABLE, SRM3_REC_TABLES_MOVED, SRM3_PAIRSUM_SEPARABLE = 1, 2, 4
SRM3_REC_COARSE_START, SRM3_REC_TABLES_INTERPOLATED = 8, 16


class srm3_info(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("max_sum_b2", ctypes.c_double),
                ("min_pure_ratio", ctypes.c_double), ("variance", ctypes.c_double),
                ("table_bytes", ctypes.c_double), ("plan_ms", ctypes.c_double),
                ("pairs", ctypes.c_int64), ("root_passes", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("tile_r", ctypes.c_int32), ("root_passes_fp32", ctypes.c_int32),
                ("interactions", ctypes.c_int32), ("fixed_point_iterations", ctypes.c_int32),
                ("diff_pairs", ctypes.c_int64), ("device_bytes", ctypes.c_double),
                ("tile_width", ctypes.c_int32), ("recursion_flags", ctypes.c_int32),
                ("coarse_fk", ctypes.c_int32), ("coarse_fw", ctypes.c_int32),
                ("coarse_launches", ctypes.c_int32), ("coarse_passes", ctypes.c_int32)]


class srm3_timings(ctypes.Structure):
    _fields_ = [("recursion_ms", ctypes.c_double), ("table_ms", ctypes.c_double),
                ("phases_ms", ctypes.c_double), ("pairsum_ms", ctypes.c_double),
                ("transform_ms", ctypes.c_double), ("recursion_passes", ctypes.c_int32),
                ("pairsum_launches", ctypes.c_int32), ("pair_terms", ctypes.c_int64),
                ("recursion_fp32_ms", ctypes.c_double), ("recursion_fp64_ms", ctypes.c_double),
                ("recursion_passes_fp32", ctypes.c_int32),
                ("recursion_passes_coarse", ctypes.c_int32), ("coarse_ms", ctypes.c_double)]


class srm3_stats_result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_double), ("power_sum", ctypes.c_double * 4),
                ("mean", ctypes.c_double), ("variance", ctypes.c_double),
                ("skewness", ctypes.c_double), ("kurtosis", ctypes.c_double),
                ("below", ctypes.c_uint64), ("above", ctypes.c_uint64)]


class SRM3Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"SRM3_ERR_{SRM3_ERR.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(build_if_needed: bool = True):
    """Load ``libsrm3.so`` (building it with nvcc when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_needed else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i32, u64p = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)
    lib.srm3_plan_create.argtypes = [ctypes.POINTER(srm3_spectrum),
                                     ctypes.POINTER(srm3_bispectrum),
                                     ctypes.POINTER(srm3_grid), ctypes.POINTER(vp)]
    lib.srm3_sample.argtypes = [vp, u64p, i32, vp]
    lib.srm3_sample_host.argtypes = [vp, u64p, i32, vp]
    lib.srm3_destroy.argtypes = [vp]
    lib.srm3_destroy.restype = None
    lib.srm3_sync.argtypes = [vp]
    lib.srm3_set_stream.argtypes = [vp, vp]
    lib.srm3_last_error.argtypes = []
    lib.srm3_last_error.restype = ctypes.c_char_p
    lib.srm3_plan_info.argtypes = [vp, ctypes.POINTER(srm3_info)]
    dp = ctypes.POINTER(ctypes.c_double)
    lib.srm3_plan_tables.argtypes = [vp, dp, dp, dp]
    lib.srm3_plan_moments.argtypes = [vp, dp, dp]
    lib.srm3_selftest_timeouts.argtypes = [ctypes.POINTER(ctypes.c_int)] * 2
    lib.srm3_phase_words.argtypes = [vp, u64p, i32, vp]
    lib.srm3_coeffs.argtypes = [vp, u64p, i32, vp]
    lib.srm3_field_from_coeffs.argtypes = [vp, vp, i32, vp]
    lib.srm3_field_from_coeffs_noalloc.argtypes = [vp, vp, i32, vp]
    lib.srm3_enable_timing.argtypes = [vp, i32]
    lib.srm3_get_timings.argtypes = [vp, ctypes.POINTER(srm3_timings), i32]
    lib.srm3_autotune.argtypes = [vp, i32, ctypes.POINTER(srm3_tune_result)]
    lib.srm3_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(vp), i32, vp, ctypes.POINTER(vp)]
    lib.srm3_batch_run.argtypes = [vp, u64p]
    lib.srm3_batch_capture.argtypes = [vp]
    lib.srm3_batch_sync.argtypes = [vp]
    lib.srm3_batch_pair_terms.argtypes = [vp]
    lib.srm3_batch_pair_terms.restype = ctypes.c_int64
    lib.srm3_set_tile_width.argtypes = [vp, i32]
    lib.srm3_batch_device_bytes.argtypes = [vp]
    lib.srm3_batch_device_bytes.restype = ctypes.c_int64
    lib.srm3_batch_destroy.argtypes = [vp]
    lib.srm3_batch_destroy.restype = None
    lib.srm3_batch_enable_timing.argtypes = [vp, i32]
    lib.srm3_batch_pairsum_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.srm3_batch_set_max_ctas.argtypes = [vp, i32]
    lib.srm3_stats_create.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.POINTER(vp)]
    lib.srm3_stats_add.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int64, vp]
    lib.srm3_stats_read.argtypes = [vp, vp, ctypes.POINTER(srm3_stats_result), u64p]
    lib.srm3_stats_reset.argtypes = [vp, vp]
    lib.srm3_stats_destroy.argtypes = [vp]
    lib.srm3_stats_destroy.restype = None
    _lib = lib
    return lib


def last_error() -> str:
    return load().srm3_last_error().decode()


def _check(rc):
    if rc != SRM3_OK:
        raise SRM3Error(rc, last_error())


def _seeds(seeds):
    a = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


# --- raw calls (same names as the C ABI) --------------------------------------

def plan_create(spectrum: srm3_spectrum, bispectrum: srm3_bispectrum, grid: srm3_grid):
    h = ctypes.c_void_p()
    _check(load().srm3_plan_create(ctypes.byref(spectrum), ctypes.byref(bispectrum),
                                   ctypes.byref(grid), ctypes.byref(h)))
    return h


def sample(plan, seeds, n, out_ptr: int):
    a, p = _seeds(seeds)
    _check(load().srm3_sample(plan, p, int(n), ctypes.c_void_p(out_ptr)))


def sample_host(plan, seeds, n, out_host_ptr: int):
    a, p = _seeds(seeds)
    _check(load().srm3_sample_host(plan, p, int(n), ctypes.c_void_p(out_host_ptr)))


def destroy(plan):
    load().srm3_destroy(plan)


def sync(plan):
    _check(load().srm3_sync(plan))


def set_stream(plan, stream_ptr: int):
    _check(load().srm3_set_stream(plan, ctypes.c_void_p(stream_ptr)))


def plan_info(plan) -> srm3_info:
    info = srm3_info()
    _check(load().srm3_plan_info(plan, ctypes.byref(info)))
    return info


def plan_tables(plan, nk, nw):
    S = np.zeros((nk, nw))
    q = np.zeros((nk, nw))
    sb2 = np.zeros((nk, nw))
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load().srm3_plan_tables(plan, S.ctypes.data_as(dp), q.ctypes.data_as(dp),
                                   sb2.ctypes.data_as(dp)))
    return S, q, sb2


def phase_words(plan, seeds, n, words_ptr: int):
    a, p = _seeds(seeds)
    _check(load().srm3_phase_words(plan, p, int(n), ctypes.c_void_p(words_ptr)))


def coeffs(plan, seeds, n, C_ptr: int):
    a, p = _seeds(seeds)
    _check(load().srm3_coeffs(plan, p, int(n), ctypes.c_void_p(C_ptr)))


def field_from_coeffs(plan, C_ptr: int, n, out_ptr: int):
    _check(load().srm3_field_from_coeffs(plan, ctypes.c_void_p(C_ptr), int(n),
                                         ctypes.c_void_p(out_ptr)))


def field_from_coeffs_noalloc(plan, C_ptr: int, n, out_ptr: int):
    """The transform through the entry point that allocates no device memory
    (its scratch is a fixed 16 MiB array per device; calls overlapping on one
    device race on it)."""
    _check(load().srm3_field_from_coeffs_noalloc(plan, ctypes.c_void_p(C_ptr), int(n),
                                                 ctypes.c_void_p(out_ptr)))


def autotune(plan, n) -> srm3_tune_result:
    r = srm3_tune_result()
    _check(load().srm3_autotune(plan, int(n), ctypes.byref(r)))
    return r


class Batch:
    """One sampling job over several plans (srm3_batch_*): uneven lattices and
    sample counts, one persistent pair-sum launch, optionally replayed from a
    captured CUDA graph.  ``outs`` are device tensors u[counts[i]][n_x][n_t]."""

    def __init__(self, plans, counts, outs, stream=None):
        m = len(plans)
        self._plans = list(plans)
        self._outs = list(outs)
        self.counts = [int(c) for c in counts]
        ph = (ctypes.c_void_p * m)(*[p.handle if hasattr(p, "handle") else p for p in plans])
        cn = (ctypes.c_int32 * m)(*self.counts)
        op = (ctypes.c_void_p * m)(*[o.data_ptr() if hasattr(o, "data_ptr") else o
                                     for o in outs])
        h = ctypes.c_void_p()
        _check(load().srm3_batch_create(ph, cn, op, m, stream, ctypes.byref(h)))
        self.handle = h

    @property
    def pair_terms(self) -> int:
        return int(load().srm3_batch_pair_terms(self.handle))

    @property
    def device_bytes(self) -> int:
        """Device memory the batch allocated itself (srm3_batch_device_bytes)."""
        return int(load().srm3_batch_device_bytes(self.handle))

    def run(self, seeds):
        a, p = _seeds(seeds)
        if len(a) != sum(self.counts):
            raise ValueError("need one seed per sample of the batch")
        _check(load().srm3_batch_run(self.handle, p))

    def capture(self):
        _check(load().srm3_batch_capture(self.handle))

    def set_max_ctas(self, n):
        _check(load().srm3_batch_set_max_ctas(self.handle, int(n)))

    def enable_timing(self, on=True):
        _check(load().srm3_batch_enable_timing(self.handle, int(bool(on))))

    def pairsum_ms(self) -> float:
        v = ctypes.c_double()
        _check(load().srm3_batch_pairsum_ms(self.handle, ctypes.byref(v)))
        return v.value

    def sync(self):
        _check(load().srm3_batch_sync(self.handle))

    def destroy(self):
        if self.handle:
            load().srm3_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


class Stats:
    """Running ensemble statistics of sampled fields on the device
    (srm3_stats_*): power sums about ``shift`` and a histogram of ``nbins``
    bins over [lo, hi).  ``add`` takes a device tensor (float32 or float64,
    any shape, contiguous); ``read`` returns mean, variance, skewness,
    kurtosis, the bin counts and the empirical PDF and CDF over the bins."""

    def __init__(self, nbins, lo, hi, shift=0.0, stream=None):
        h = ctypes.c_void_p()
        _check(load().srm3_stats_create(int(nbins), float(lo), float(hi), float(shift),
                                        ctypes.byref(h)))
        self.handle = h
        self.nbins, self.lo, self.hi = int(nbins), float(lo), float(hi)
        self.stream = stream

    def add(self, u, precision=None, count=None):
        if precision is None:
            precision = SRM3_FP64 if str(getattr(u, "dtype", "")) == "torch.float64" else SRM3_FP32
        if count is None:
            count = u.numel()
        ptr = u.data_ptr() if hasattr(u, "data_ptr") else int(u)
        _check(load().srm3_stats_add(self.handle, ptr, int(precision), int(count), self.stream))

    def read(self):
        import numpy as np
        r = srm3_stats_result()
        hist = np.zeros(self.nbins, dtype=np.uint64)
        _check(load().srm3_stats_read(self.handle, self.stream, ctypes.byref(r),
                                      hist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        width = (self.hi - self.lo) / self.nbins
        n = r.count
        cum = np.cumsum(hist.astype(np.float64)) + float(r.below)
        return {
            "count": n, "power_sum": list(r.power_sum), "mean": r.mean,
            "variance": r.variance, "skewness": r.skewness, "kurtosis": r.kurtosis,
            "below": int(r.below), "above": int(r.above), "hist": hist,
            "edges": self.lo + width * np.arange(self.nbins + 1),
            "pdf": hist / (n * width) if n > 0 else hist.astype(np.float64),
            "cdf": cum / n if n > 0 else cum,
        }

    def reset(self):
        _check(load().srm3_stats_reset(self.handle, self.stream))

    def destroy(self):
        if self.handle:
            load().srm3_stats_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


def enable_timing(plan, on: bool):
    _check(load().srm3_enable_timing(plan, int(bool(on))))


def get_timings(plan, reset: bool = False) -> srm3_timings:
    t = srm3_timings()
    _check(load().srm3_get_timings(plan, ctypes.byref(t), int(bool(reset))))
    return t


# --- convenience wrapper -------------------------------------------------------

_PREC = {"fp32": SRM3_FP32, "fp64": SRM3_FP64}
_STOR = {"auto": SRM3_STORAGE_AUTO, "table": SRM3_STORAGE_TABLE,
         "recompute": SRM3_STORAGE_RECOMPUTE, "tuned": SRM3_STORAGE_TUNED}


@dataclass
class Plan:
    """A plan built from a workload description (see ``workloads.Workload``)."""
    handle: ctypes.c_void_p
    nk: int
    nw: int
    nx: int
    nt: int
    precision: str

    @classmethod
    def create(cls, wl, *, precision=None, storage=None, stream=None, table=None,
               eps=None, target=None, budget_bytes=0.0, mixed=None, rows=None):
        prec = precision or wl.precision
        sp = srm3_spectrum()
        keep = None
        if table is None:
            sp.kind = SRM3_SPECTRUM_KAIMAL_LORENTZIAN
            sp.U, sp.z, sp.z0, sp.k_vk, sp.lam = wl.U, wl.z, wl.z0, wl.k_vk, wl.lam
        else:
            keep = np.ascontiguousarray(table, dtype=np.float64)
            sp.kind = SRM3_SPECTRUM_TABLE
            sp.table = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        bs = srm3_bispectrum()
        bs.kind = SRM3_BISPECTRUM_GAUSS_ENVELOPE
        env = env_b = None
        if wl.envelope != "gauss":
            ta, tb = wl.envelope_tables()
            env = np.ascontiguousarray(ta, dtype=np.float64)
            bs.kind = SRM3_BISPECTRUM_SEPARABLE
            bs.env_table = env.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            if tb is not None:
                env_b = np.ascontiguousarray(tb, dtype=np.float64)
                bs.env_table_b = env_b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        tgt = wl.target if target is None else target
        if eps is None and target is None and getattr(wl, "eps", 0.0) > 0.0:
            eps = wl.eps
        if eps is not None:
            bs.target_max_sum_b2, bs.eps = 0.0, float(eps)
        else:
            bs.target_max_sum_b2 = float(tgt)
        bs.sigma_g, bs.beta = wl.sigma_g, wl.beta
        mx = getattr(wl, "interactions", "sum") == "mixed" if mixed is None else bool(mixed)
        bs.interactions = SRM3_INTERACTIONS_MIXED if mx else SRM3_INTERACTIONS_SUM
        g = srm3_grid()
        g.n_kappa, g.n_omega = wl.n_kappa, wl.n_omega
        g.kappa_u, g.omega_u = wl.kappa_u, wl.omega_u
        g.n_x, g.n_t = wl.n_x, wl.n_t
        g.precision = _PREC[prec]
        g.storage = _STOR[storage or wl.storage]
        g.stream = stream
        g.table_budget_bytes = float(budget_bytes)
        if rows is not None:  # one shard: lattice rows [rows[0], rows[1])
            g.row_begin, g.row_end = int(rows[0]), int(rows[1])
        h = plan_create(sp, bs, g)
        del keep, env, env_b
        return cls(h, wl.n_kappa, wl.n_omega, wl.n_x, wl.n_t, prec)

    def info(self) -> srm3_info:
        return plan_info(self.handle)

    def set_tile_width(self, width: int):
        """FP32 pair-sum work unit: 32 or 16 outputs (srm3_set_tile_width)."""
        _check(load().srm3_set_tile_width(self.handle, int(width)))

    def tables(self):
        return plan_tables(self.handle, self.nk, self.nw)

    def moments(self):
        """(variance, third moment) of u, exact (srm3_plan_moments)."""
        v, m3 = ctypes.c_double(), ctypes.c_double()
        _check(load().srm3_plan_moments(self.handle, ctypes.byref(v), ctypes.byref(m3)))
        return v.value, m3.value

    def _torch_dtype(self):
        import torch
        return torch.float32 if self.precision == "fp32" else torch.float64

    def sample(self, seeds, out=None):
        import torch
        n = len(seeds)
        if out is None:
            out = torch.empty((n, self.nx, self.nt), dtype=self._torch_dtype(), device="cuda")
        sample(self.handle, seeds, n, out.data_ptr())
        return out

    def coeffs(self, seeds):
        import torch
        n = len(seeds)
        C = torch.empty((n, 2, self.nk, self.nw, 2), dtype=self._torch_dtype(), device="cuda")
        coeffs(self.handle, seeds, n, C.data_ptr())
        return C

    def field_from_coeffs(self, C):
        import torch
        n = C.shape[0]
        out = torch.empty((n, self.nx, self.nt), dtype=self._torch_dtype(), device="cuda")
        field_from_coeffs(self.handle, C.data_ptr(), n, out.data_ptr())
        return out

    def phase_words(self, seeds):
        import torch
        n = len(seeds)
        w = torch.empty((n, 2, self.nk, self.nw), dtype=torch.int32, device="cuda")
        phase_words(self.handle, seeds, n, w.data_ptr())
        return w

    def sync(self):
        sync(self.handle)

    def destroy(self):
        if self.handle:
            destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()
