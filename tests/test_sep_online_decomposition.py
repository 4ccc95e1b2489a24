"""The online FFT form of the separable recursion's bulk, checked on the CPU.

For g = a_i a_j b_k the pair sums of a plane are a 2-D self-convolution of h
over (level, kk).  The recursion pass replaces its bulk phases by a divide and
conquer over levels: before each 16-level block [D, D + 16) one product with
L = 16 2^{v2(D/16)}, l0 = D - L adds, on a cyclic 2L x Nc grid, the ordered
pairs with one level in [l0, D) and the other in [0, 2L) (both in [0, L) when
l0 = 0); the block then adds half the diagonal term and its fringe (pairs
with a part in [D, d)).  This test restates that schedule in numpy -- every
product fed only the levels below its block -- and checks that it equals the
direct unordered pair sums on lattices of several shapes."""
import numpy as np
import pytest

BL = 16


def _direct(h):
    nk, nw = h.shape
    out = np.zeros_like(h)
    for kk in range(nk):
        for kw in range(nw):
            s = 0.0
            for ik in range(kk + 1):
                for iw in range(kw + 1):
                    jk, jw = kk - ik, kw - iw
                    if (ik, iw) == (0, 0) or (jk, jw) == (0, 0) or (ik, iw) > (jk, jw):
                        continue
                    s += h[ik, iw] * h[jk, jw]
            out[kk, kw] = s
    return out


def _online(h):
    nk, nw = h.shape
    nlev = nk + nw - 1
    lev = np.add.outer(np.arange(nk), np.arange(nw))
    acc = np.zeros_like(h)
    out = np.full_like(h, np.nan)
    l2max = max([2 * BL * ((D // BL) & -(D // BL)) for D in range(BL, nlev, BL)] + [2])
    nc = 2
    while nc < nk + min(l2max, nk) - 1:
        nc *= 2

    def hget(known, d, kk):
        kw = d - kk
        if d == 0 or kk >= nk or kw < 0 or kw >= nw:
            return 0.0
        v = known[kk, kw]
        assert not np.isnan(v), "a product read a level at or above its block"
        return v

    for D in range(BL, nlev, BL):
        known = np.where(lev < D, h, np.nan)
        L = BL * ((D // BL) & -(D // BL))
        l0, L2 = D - L, 2 * L
        z = np.zeros((L2, nc), complex)
        for o in range(L2):
            for kk in range(nc):
                re = hget(known, l0 + o, kk) if o < L else 0.0
                im = hget(known, o, kk) if l0 > 0 else 0.0
                z[o, kk] = re + 1j * im
        F = np.fft.ifft2(z) * z.size  # the e^{+2 pi i} direction, unnormalised
        G = np.fft.ifft2(F * F) * z.size
        for o in range(L, L2):
            d = l0 + o
            if d >= nlev:
                continue
            for kk in range(max(0, d - nw + 1), min(d, nk - 1) + 1):
                v = G[(-o) % L2, (-kk) % nc] / (L2 * nc)
                acc[kk, d - kk] += 0.5 * (v.imag if l0 > 0 else v.real)
        for d in range(D, min(D + BL, nlev)):
            for kk in range(max(0, d - nw + 1), min(d, nk - 1) + 1):
                kw = d - kk
                s = acc[kk, kw]
                if kk % 2 == 0 and kw % 2 == 0:
                    s += 0.5 * h[kk // 2, kw // 2] ** 2
                for l in range(1, d - D + 1):  # fringe: a part in [D, d)
                    for lk in range(l + 1):
                        lw = l - lk
                        if kk - lk >= 0 and kw - lw >= 0:
                            s += h[lk, lw] * h[kk - lk, kw - lw]
                out[kk, kw] = s
    return out, lev >= BL


@pytest.mark.parametrize("nk,nw", [(24, 37), (40, 70), (9, 40), (70, 20)])
def test_online_schedule_equals_direct_pair_sums(nk, nw):
    rng = np.random.default_rng(nk * 1000 + nw)
    h = rng.uniform(0.5, 2.0, (nk, nw))
    h[0, 0] = 0.0
    got, mask = _online(h)
    ref = _direct(h)
    assert not np.isnan(got[mask]).any()
    np.testing.assert_allclose(got[mask], ref[mask], rtol=0, atol=1e-12 * np.abs(ref).max())
