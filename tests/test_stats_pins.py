"""Pins of the oracle's sample statistics (Sec. 6: sample mean, variance,
skewness; empirical PDF/CDF) to closed forms: a sinusoid sampled over whole
periods, the centres of a uniform grid, and a two-point distribution."""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("offset", [0.0, 5.0])
def test_sinusoid_moments(offset):
    # sum over whole periods: <sin> = <sin^3> = 0, <sin^2> = 1/2, <sin^4> = 3/8
    n, a = 4096, 3.0
    u = offset + a * np.sin(2 * np.pi * np.arange(n) / n)
    for shift in (0.0, offset):
        r = oracle.field_stats(u, 8, -4.0 + offset, 4.0 + offset, shift=shift)
        assert r["count"] == n
        assert r["mean"] == pytest.approx(offset, abs=1e-12)
        assert r["variance"] == pytest.approx(a * a / 2, rel=1e-12)
        assert abs(r["skewness"]) < 1e-12
        assert r["kurtosis"] == pytest.approx(1.5, rel=1e-11)
        assert r["below"] == 0 and r["above"] == 0
        assert int(r["hist"].sum()) == n


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_uniform_grid_moments_and_bins(dtype):
    # centres (m + 1/2)/N of N equal cells: discrete uniform on N points
    n, nb = 1024, 16
    u = ((np.arange(n) + 0.5) / n).astype(dtype)
    r = oracle.field_stats(u, nb, 0.0, 1.0)
    assert r["mean"] == pytest.approx(0.5, abs=1e-15)
    assert r["variance"] == pytest.approx((n * n - 1) / (12.0 * n * n), rel=1e-13)
    assert abs(r["skewness"]) < 1e-12
    kurt = 3.0 - 6.0 * (n * n + 1) / (5.0 * (n * n - 1))
    assert r["kurtosis"] == pytest.approx(kurt, rel=1e-12)
    assert r["hist"].tolist() == [n // nb] * nb
    # out of range: below lo, exactly hi, and a NaN count apart
    extra = np.array([-0.1, 1.0, np.nan], dtype=dtype)
    r2 = oracle.field_stats(np.concatenate([u, extra]), nb, 0.0, 1.0)
    assert r2["below"] == 1 and r2["above"] == 2
    assert r2["hist"].tolist() == [n // nb] * nb


def test_two_point_distribution():
    # P(u = 1) = p: skewness (1 - 2p)/sqrt(pq), kurtosis (1 - 3pq)/(pq)
    u = np.concatenate([np.zeros(300), np.ones(100)])
    p, q = 0.25, 0.75
    r = oracle.field_stats(u, 2, 0.0, 2.0, shift=0.1)
    assert r["mean"] == pytest.approx(p, rel=1e-14)
    assert r["variance"] == pytest.approx(p * q, rel=1e-13)
    assert r["skewness"] == pytest.approx((1 - 2 * p) / math.sqrt(p * q), rel=1e-12)
    assert r["kurtosis"] == pytest.approx((1 - 3 * p * q) / (p * q), rel=1e-12)
    assert r["hist"].tolist() == [300, 100]
