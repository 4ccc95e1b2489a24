"""Device sample statistics (srm3_stats_*, Sec. 6: sample moments and the
empirical PDF/CDF of simulated waves) against the oracle's definitions
(pinned in test_stats_pins.py), and the sampled skewness of the method
against its exact third moment.

Tolerances: bin counts and out-of-range counts bit-exact (the bin decision is
taken in the input's precision on both sides); power sums of FP32 input
within 2e-6 of sum |u - shift|^p (each thread sums 16 values in FP32 before
FP64: at most 16 roundings of 2^-24 relative each), FP64 input within 1e-12
of it.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2310_03979_gb300 import srm3
from paper_2310_03979_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _check_against_oracle(res, ref, u64, shift, rel):
    assert res["count"] == ref["count"]
    np.testing.assert_array_equal(res["hist"], ref["hist"])
    assert res["below"] == ref["below"] and res["above"] == ref["above"]
    d = np.abs(u64 - shift)
    for p in range(4):
        scale = float(np.sum(d ** (p + 1)))
        assert abs(res["power_sum"][p] - ref["power_sum"][p]) <= rel * scale + 1e-300


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_stats_match_oracle_in_chunks(dtype):
    g = torch.Generator().manual_seed(7)
    n = 3 * 65536 + 7  # a ragged tail after the 16-byte vectors
    base = torch.randn(n, generator=g, dtype=torch.float64) * 18.0
    torch.manual_seed(11)
    skewed = torch.distributions.Gamma(2.0, 0.1).sample((n,)) - 20.0
    u = torch.cat([base, skewed.to(torch.float64)]).to(dtype)
    u[11] = 1e6
    nbins, lo, hi, shift = 257, -80.0, 120.0, 0.5
    ud = u.cuda()
    # three chunks, each starting on a 16-byte boundary
    cut = [0, 4 * 12345, 4 * 70001, ud.numel()]
    with srm3.Stats(nbins, lo, hi, shift) as st:
        for a, b in zip(cut[:-1], cut[1:]):
            st.add(ud[a:b])
        res = st.read()
    un = u.numpy()
    ref = oracle.field_stats(un, nbins, lo, hi, shift)
    rel = 2e-6 if dtype == torch.float32 else 1e-12
    _check_against_oracle(res, ref, un.astype(np.float64), shift, rel)
    assert res["above"] >= 1  # the large value


def test_stats_deterministic_and_reset():
    g = torch.Generator().manual_seed(3)
    u = (torch.randn(1 << 20, generator=g) * 5).cuda()
    with srm3.Stats(64, -20, 20) as st:
        st.add(u)
        r1 = st.read()
        st.reset()
        st.add(u)
        r2 = st.read()
        st.add(u[:0])  # count 0: no-op
        r3 = st.read()
    assert r1["power_sum"] == r2["power_sum"] == r3["power_sum"]
    np.testing.assert_array_equal(r1["hist"], r2["hist"])
    assert r1["cdf"][-1] == pytest.approx(1.0 - r1["above"] / r1["count"])


def test_stats_edges_and_errors():
    # values on bin edges: the FP32 decision, as the oracle takes it
    lo, hi, nb = -1.0, 1.0, 8
    edges = np.float32(lo) + np.arange(nb + 1, dtype=np.float32) * np.float32((hi - lo) / nb)
    u = np.concatenate([edges, np.nextafter(edges, np.float32(-2)),
                        np.nextafter(edges, np.float32(2))]).astype(np.float32)
    u = np.concatenate([u, np.array([np.nan, 5.0, -5.0], np.float32)])
    with srm3.Stats(nb, lo, hi) as st:
        st.add(torch.from_numpy(u).cuda())
        res = st.read()
    ref = oracle.field_stats(u, nb, lo, hi)
    np.testing.assert_array_equal(res["hist"], ref["hist"])
    assert (res["below"], res["above"]) == (ref["below"], ref["above"])
    with srm3.Stats(1, 0, 1) as st:  # one bin
        st.add(torch.full((40,), 0.5, device="cuda"))
        assert st.read()["hist"].tolist() == [40]
        ud = torch.zeros(8, device="cuda")
        with pytest.raises(srm3.SRM3Error):
            st.add(ud[1:], count=4)  # not 16-byte aligned
    with pytest.raises(srm3.SRM3Error):
        srm3.Stats(0, 0, 1)
    with pytest.raises(srm3.SRM3Error):
        srm3.Stats(4, 1, 1)


@pytest.mark.parametrize("envelope", ["gauss", "sum"])
def test_sampled_fields_stats_and_skewness(envelope):
    """Fields of a plan: device statistics equal the oracle's on the same
    fields, and the sample skewness over 512 samples agrees with the exact
    E[u^3] / E[u^2]^1.5 of the discrete model within five standard errors
    of the mean over 16 independent groups of samples.  "sum": the envelope
    of i + j alone of the bridge bispectrum (Sec. 5), sampled through the
    separable FFT forms of the recursion and the pair sum."""
    wl = W.small_case(nk=32, nw=32, nx=64, nt=64, seeds=(1,), target=0.7)
    if envelope != "gauss":
        import dataclasses
        wl = dataclasses.replace(wl, envelope=envelope)
    groups, per = 16, 32
    with srm3.Plan.create(wl) as p:
        var, m3 = p.moments()
        sig = math.sqrt(var)
        skews, vars_ = [], []
        for gi in range(groups):
            seeds = [1000 * gi + j + 1 for j in range(per)]
            u = p.sample(seeds)
            with srm3.Stats(101, -6 * sig, 6 * sig) as st:
                st.add(u)
                r = st.read()
            if gi == 0:
                un = u.cpu().numpy()
                ref = oracle.field_stats(un, 101, -6 * sig, 6 * sig)
                _check_against_oracle(r, ref, un.astype(np.float64), 0.0, 2e-6)
            skews.append(r["skewness"])
            vars_.append(r["variance"])
    exact = m3 / var ** 1.5
    s, se = np.mean(skews), np.std(skews, ddof=1) / math.sqrt(groups)
    assert exact > 0.05
    assert abs(s - exact) < 5 * se, (s, exact, se)
    v, sev = np.mean(vars_), np.std(vars_, ddof=1) / math.sqrt(groups)
    assert abs(v - var) < 5 * sev, (v, var, sev)
