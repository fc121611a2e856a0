"""Pins of the oracle's log-matched filter, peak picking and initial cloud."""
import numpy as np
import pytest

import scenes


def _irf(orc, kind="gauss"):
    g = scenes.gaussian_irf(3.0, 12) if kind == "gauss" else scenes.gamma_irf(3, 5, 80)
    return orc.OIrf(g.samples, g.origin)


def test_lmf_kernel_values(orc):
    irf = _irf(orc, "gamma")
    k = orc.lmf_kernel(irf, 1e-3, 5)
    assert k.min() >= 0
    d = float(np.float32(1e-3))
    assert k[irf.origin] == int(np.rint(32 * np.log1p(1.0 / d)))
    assert k.max() == k[irf.origin]
    assert k.max() < 256           # fits the bf16 significand


@pytest.mark.parametrize("t0,c", [(40, 1), (41, 7), (2, 3), (126, 2)])
def test_lmf_of_a_delta_is_the_reflected_kernel(orc, t0, c):
    irf = _irf(orc, "gauss")
    kern = orc.lmf_kernel(irf, 1e-3, 5)
    z = np.zeros(128, np.uint16)
    z[t0] = c
    y, wc = orc.lmf(z, kern, irf.origin)
    for tau in range(128):
        s = t0 - tau + irf.origin
        want = c * kern[s] if 0 <= s < len(kern) else 0
        assert y[tau] == want
        assert wc[tau] == (c if 0 <= s < len(kern) else 0)


def test_lmf_is_linear_and_shift_equivariant(orc):
    rng = np.random.default_rng(0)
    irf = _irf(orc, "gamma")
    kern = orc.lmf_kernel(irf, 1e-3, 5)
    a = rng.poisson(0.3, 400).astype(np.uint16)
    b = rng.poisson(0.3, 400).astype(np.uint16)
    ya, _ = orc.lmf(a, kern, irf.origin)
    yb, _ = orc.lmf(b, kern, irf.origin)
    yab, _ = orc.lmf(a + b, kern, irf.origin)
    assert np.array_equal(ya + yb, yab)
    sh = np.zeros(400, np.uint16)
    sh[100:300] = a[100:300]
    sh2 = np.roll(sh, 37)
    y1, _ = orc.lmf(sh, kern, irf.origin)
    y2, _ = orc.lmf(sh2, kern, irf.origin)
    assert np.array_equal(np.roll(y1, 37)[150:350], y2[150:350])


def test_peaks_of_separated_returns(orc):
    """Three well separated noise-free returns: peaks sit at the true integer
    depths, in depth order, whatever their relative strength; only the K
    strongest survive when K is smaller."""
    irf = _irf(orc, "gauss")
    kern = orc.lmf_kernel(irf, 1e-3, 5)
    t = 300
    z = np.zeros(t, np.uint16)
    for d, amp in ((50, 9), (140, 30), (230, 15)):
        for s in range(len(irf.h)):
            z[d + s - irf.origin] += int(round(amp * irf.h[s] * 10))
    y, wc = orc.lmf(z, kern, irf.origin)
    assert list(orc.peaks(y, wc, 6, 2, 3)) == [50, 140, 230]
    assert list(orc.peaks(y, wc, 6, 2, 2)) == [140, 230]
    assert list(orc.peaks(y, wc, 6, 2, 1)) == [140]
    # shift equivariance and count scaling
    z2 = np.roll(z, 11)
    y2, wc2 = orc.lmf(z2, kern, irf.origin)
    assert list(orc.peaks(y2, wc2, 6, 2, 3)) == [61, 151, 241]
    y3, wc3 = orc.lmf((z * 3).astype(np.uint16), kern, irf.origin)
    assert list(orc.peaks(y3, wc3, 6, 2, 3)) == [50, 140, 230]


def test_peaks_tie_rules_and_thresholds(orc):
    y = np.zeros(40, np.int64)
    wc = np.full(40, 5, np.int64)
    y[10] = y[11] = 7              # plateau: the earlier bin wins
    y[30] = 4
    assert list(orc.peaks(y, wc, 3, 2, 3)) == [10, 30]
    wc[30] = 1                      # too few photons in its window
    assert list(orc.peaks(y, wc, 3, 2, 3)) == [10]
    y2 = np.zeros(40, np.int64)
    y2[[5, 20, 35]] = 6            # equal heights: K=2 keeps the two earliest
    assert list(orc.peaks(y2, wc, 3, 1, 2)) == [5, 20]
    assert len(orc.peaks(np.zeros(40, np.int64), wc, 3, 0, 3)) == 0


def test_init_closed_form(orc):
    """One strong return plus a known number of background counts: t0 is the
    return's bin, b0 = outside counts / outside bins, r0 = window counts - b0 |window|."""
    irf = _irf(orc, "gauss")
    t = 200
    z = np.zeros((1, 1, t), np.uint16)
    for s in range(len(irf.h)):
        z[0, 0, 100 + s - irf.origin] += int(round(40 * irf.h[s] * 5))
    outside = [3, 40, 150, 190]     # farther apart than one IRF window
    z[0, 0, outside] += 1
    prm = scenes.make_params(scenes.small_random(2, 2, t), k_max=2)
    st = orc.init(z, None, irf, prm)
    assert st.alive[0, 0, 0] == 1 and st.alive[1, 0, 0] == 0
    assert st.t[0, 0, 0] == 100.0
    win = len(irf.h)
    b0 = len(outside) / (t - win)
    assert abs(st.b[0, 0] - b0) < 1e-15
    wcount = int(z[0, 0, 100 - irf.origin:100 - irf.origin + win].sum())
    assert abs(st.r[0, 0, 0] - (wcount - b0 * win)) < 1e-12


def test_init_empty_and_dead_pixels(orc):
    irf = _irf(orc, "gauss")
    prm = scenes.make_params(scenes.small_random(2, 2, 64), k_max=2)
    z = np.zeros((2, 2, 64), np.uint16)
    z[1, 1, 30] = 9
    gain = np.ones((2, 2))
    gain[1, 1] = 0.0
    st = orc.init(z, gain, irf, prm)
    assert st.alive.sum() == 0
    np.testing.assert_allclose(st.b, np.float32(prm["b_floor"]))


def test_peaks_match_brute_force_on_random_tiny_inputs(orc):
    """The peak picker against its definition evaluated by brute force: the
    admissible positions (positive filter value, enough photons in the IRF
    window, strictly above every value up to sep bins earlier and at least every
    value up to sep bins later, the histogram ends cutting the neighbourhood),
    the K best of them under (value descending, bin ascending) by a full sort,
    reported by increasing bin.  Small integer values give many plateaus and
    ties."""
    rng = np.random.default_rng(11)
    for _ in range(400):
        t = int(rng.integers(1, 41))
        y = rng.integers(-2, 7, t).astype(np.int64)
        wc = rng.integers(0, 6, t).astype(np.int64)
        sep = int(rng.integers(0, 5))
        thr = int(rng.integers(0, 5))
        kmax = int(rng.integers(1, 5))
        adm = [tau for tau in range(t)
               if y[tau] > 0 and wc[tau] >= thr
               and all(y[tau] > y[q] for q in range(max(0, tau - sep), tau))
               and all(y[tau] >= y[q] for q in range(tau + 1, min(t, tau + sep + 1)))]
        want = sorted(sorted(adm, key=lambda tau: (-y[tau], tau))[:kmax])
        assert list(orc.peaks(y, wc, sep, thr, kmax)) == want, (t, sep, thr, kmax, y.tolist(), wc.tolist())
