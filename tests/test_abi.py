"""The C ABI library: it loads without a GPU, exports every call that
include/srm3.h declares, and rejects bad arguments on the host before any
CUDA work (CPU only: no compute call runs here)."""
import ctypes
import math
import os
import re

import pytest

from paper_2310_03979_gb300 import srm3
from paper_2310_03979_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "srm3.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(srm3_[a-z_]+)\s*\(", hdr)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("srm3_plan_create", "srm3_sample", "srm3_destroy"):
        assert n in names
    assert set(names) == set(srm3.EXPORTED)


def test_library_exports_every_declared_symbol():
    lib = srm3.load()
    for name in _declared():
        assert hasattr(lib, name), name
    assert lib.srm3_last_error() is not None


def _structs(wl, **kw):
    sp = srm3.srm3_spectrum(kind=0, U=wl.U, z=wl.z, z0=wl.z0, k_vk=wl.k_vk, lam=wl.lam)
    bs = srm3.srm3_bispectrum(kind=0, target_max_sum_b2=wl.target, sigma_g=wl.sigma_g)
    g = srm3.srm3_grid(n_kappa=wl.n_kappa, n_omega=wl.n_omega, kappa_u=wl.kappa_u,
                       omega_u=wl.omega_u, n_x=wl.n_x, n_t=wl.n_t, precision=0, storage=0)
    for k, v in kw.items():
        for s in (sp, bs, g):
            if hasattr(s, k):
                setattr(s, k, v)
    return sp, bs, g


@pytest.mark.parametrize("field,value,code", [
    ("n_x", 48, -2),            # not a power of two
    ("n_t", 32, -2),            # n_t < 2 n_omega - 1
    ("n_x", 16, -2),            # n_x < n_kappa
    ("n_kappa", 0, -1),
    ("kappa_u", -1.0, -1),
    ("precision", 7, -1),
    ("storage", 9, -1),
    ("sigma_g", 0.0, -1),
    ("target_max_sum_b2", 1.0, -1),
    ("U", 0.0, -1),
])
def test_host_validation(field, value, code):
    wl = W.small_case(nk=24, nw=20, nx=64, nt=64)
    sp, bs, g = _structs(wl, **{field: value})
    h = ctypes.c_void_p(123)
    rc = srm3.load().srm3_plan_create(ctypes.byref(sp), ctypes.byref(bs), ctypes.byref(g),
                                      ctypes.byref(h))
    assert rc == code
    assert h.value is None
    assert srm3.last_error() != ""


def test_null_and_noop_calls():
    lib = srm3.load()
    assert lib.srm3_plan_create(None, None, None, None) == -1
    assert lib.srm3_sample(None, None, 0, None) == -1
    lib.srm3_destroy(None)
    assert lib.srm3_plan_info(None, None) == -1
    wl = W.small_case()
    sp, bs, g = _structs(wl)
    g.precision, g.storage = 1, 1          # FP64 plans have no W table
    h = ctypes.c_void_p()
    assert lib.srm3_plan_create(ctypes.byref(sp), ctypes.byref(bs), ctypes.byref(g),
                                ctypes.byref(h)) == -8


def test_separable_envelope_validation():
    """SEPARABLE needs a finite, non-negative env_table (env_table_b may be
    NULL, but if given it obeys the same rules); an unknown kind is refused.
    All checked on the host before any device work."""
    import numpy as np
    lib = srm3.load()
    wl = W.small_case(nk=24, nw=20, nx=64, nt=64)
    good = np.ones((24, 20))
    bad = good.copy()
    bad[3, 4] = -1.0
    nan = good.copy()
    nan[0, 1] = np.nan
    dp = ctypes.POINTER(ctypes.c_double)
    for a, b in [(None, None), (bad, None), (nan, None), (good, bad), (good, nan)]:
        sp, bs, g = _structs(wl)
        bs.kind = srm3.SRM3_BISPECTRUM_SEPARABLE
        if a is not None:
            bs.env_table = np.ascontiguousarray(a).ctypes.data_as(dp)
        if b is not None:
            bs.env_table_b = np.ascontiguousarray(b).ctypes.data_as(dp)
        h = ctypes.c_void_p(123)
        rc = lib.srm3_plan_create(ctypes.byref(sp), ctypes.byref(bs), ctypes.byref(g),
                                  ctypes.byref(h))
        assert rc == -1 and h.value is None
        assert b"env_table" in lib.srm3_last_error()
    sp, bs, g = _structs(wl)
    bs.kind = 7
    h = ctypes.c_void_p(123)
    assert lib.srm3_plan_create(ctypes.byref(sp), ctypes.byref(bs), ctypes.byref(g),
                                ctypes.byref(h)) == -1
    assert h.value is None
