"""Pins of the oracle's denoisers: APSS, intensity low-pass, background low-pass."""
import numpy as np
import pytest

import scenes


def _params(**over):
    p = scenes.make_params(scenes.small_random(4, 4, 64))
    p.update(dict(k_max=1))
    p.update(over)
    return p


def _cloud(orc, depth):
    k = 1 if depth.ndim == 2 else depth.shape[0]
    d = depth.reshape(k, *depth.shape[-2:])
    st = orc.new_state(k, d.shape[1], d.shape[2])
    st.t[:] = d
    st.alive[:] = np.isfinite(d)
    st.t[~np.isfinite(d)] = 0
    st.r[:] = 1.0
    st.b[:] = 0.01
    return st


@pytest.mark.parametrize("gi,gj", [(0.0, 0.0), (0.4, -0.3), (1.5, 2.0), (-4.0, 3.0)])
def test_apss_leaves_exact_planes_fixed(orc, gi, gj):
    """APSS reproduces planes (Guennebaud & Gross: spheres and planes are exact)."""
    h, w = 11, 13
    prm = _params(pixel_pitch=8.0, apss_radius=20.0, int_radius=20.0)
    i, j = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    depth = 500.0 + gi * prm["pixel_pitch"] * i + gj * prm["pixel_pitch"] * j
    st = _cloud(orc, depth)
    orc.apss(h, w, 2000, prm, st)
    np.testing.assert_allclose(st.t[0], depth, atol=1e-9)


@pytest.mark.parametrize("radius", [60.0, 150.0])
def test_apss_leaves_exact_spheres_fixed(orc, radius):
    h, w = 15, 15
    prm = _params(pixel_pitch=4.0, apss_radius=12.0)
    i, j = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    x, y = prm["pixel_pitch"] * (j - 7.2), prm["pixel_pitch"] * (i - 6.9)
    depth = 900.0 - np.sqrt(radius ** 2 - x ** 2 - y ** 2)
    st = _cloud(orc, depth)
    orc.apss(h, w, 2000, prm, st)
    np.testing.assert_allclose(st.t[0], depth, atol=1e-9)


def test_apss_commutes_with_depth_shift_and_smooths_noise(orc):
    rng = np.random.default_rng(0)
    h, w = 12, 12
    prm = _params()
    i, j = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    true = 300 + 3.0 * i - 2.0 * j
    noisy = true + rng.normal(0, 2.0, (h, w))
    a = _cloud(orc, noisy)
    b = _cloud(orc, noisy + 123.25)
    orc.apss(h, w, 2000, prm, a)
    orc.apss(h, w, 2000, prm, b)
    np.testing.assert_allclose(b.t - 123.25, a.t, atol=1e-9)
    assert np.std(a.t[0] - true) < 0.7 * np.std(noisy - true)


def test_apss_ignores_other_surfaces_and_degenerate_windows(orc):
    """A second surface farther than the radius does not move the first, and a
    one-row image (collinear neighbours) is left unchanged."""
    h, w = 9, 9
    prm = _params(k_max=2)
    i, j = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    front = 400 + 2.0 * i + 1.0 * j
    back = 400 + 200 + 0.0 * i + np.random.default_rng(1).normal(0, 3, (h, w))
    st = _cloud(orc, np.stack([front, back]))
    orc.apss(h, w, 2000, prm, st)
    np.testing.assert_allclose(st.t[0], front, atol=1e-9)
    row = _cloud(orc, np.array([[100.0, 103.0, 99.0, 101.0, 104.0, 98.0, 102.0]]))
    before = row.t.copy()
    orc.apss(1, 7, 2000, prm, row)
    assert np.array_equal(row.t, before)


def test_intensity_lowpass_constant_and_pruning(orc):
    h, w = 6, 7
    prm = _params(r_min=0.5)
    st = _cloud(orc, 200 + np.random.default_rng(2).normal(0, 1, (h, w)))
    st.r[:] = 3.25
    orc.int_lowpass(h, w, prm, st)
    np.testing.assert_allclose(st.r, 3.25, rtol=1e-14)
    assert st.alive.all()
    # an isolated low point is averaged with its neighbours; a uniformly low
    # patch falls below r_min and is removed
    st.r[:] = 0.4
    orc.int_lowpass(h, w, prm, st)
    assert not st.alive.any()


def test_intensity_lowpass_stays_on_its_surface(orc):
    h, w = 6, 6
    prm = _params(k_max=2)
    st = _cloud(orc, np.stack([np.full((h, w), 100.0), np.full((h, w), 600.0)]))
    st.r[0] = 1.0
    st.r[1] = 9.0
    orc.int_lowpass(h, w, prm, st)
    np.testing.assert_allclose(st.r[0], 1.0)
    np.testing.assert_allclose(st.r[1], 9.0)


@pytest.mark.parametrize("h,w,sigma,rad", [(8, 8, 1.0, 3), (5, 7, 0.8, 2), (8, 8, 2.0, 6)])
def test_background_lowpass_equals_fft_filter(orc, h, w, sigma, rad):
    """Periodic Gaussian filtering equals multiplying the 2-D DFT of the image by
    the DFT of the (wrapped) kernel -- the FFT denoiser of the paper."""
    rng = np.random.default_rng(4)
    b = rng.uniform(0, 1, (h, w))
    prm = _params(bkg_mode=1, bkg_sigma=sigma, bkg_radius=rad)
    d = np.arange(-rad, rad + 1)
    k1 = np.exp(-d.astype(float) ** 2 / (2 * np.float32(sigma) ** 2))
    k1 /= k1.sum()
    ker = np.zeros((h, w))
    for a, ka in zip(d, k1):
        for c, kc in zip(d, k1):
            ker[a % h, c % w] += ka * kc
    want = np.real(np.fft.ifft2(np.fft.fft2(b) * np.fft.fft2(ker)))
    got = b.copy()
    orc.bkg_lowpass(h, w, prm, got)
    np.testing.assert_allclose(got, want, atol=1e-12)
    const = np.full((h, w), 0.37)
    orc.bkg_lowpass(h, w, prm, const)
    np.testing.assert_allclose(const, 0.37, rtol=1e-14)
    ident = b.copy()
    orc.bkg_lowpass(h, w, _params(bkg_mode=0), ident)
    assert np.array_equal(ident, b)


def test_apss_matches_weighted_least_squares_sphere_by_lstsq(orc):
    """APSS on a generic cloud (a curved, noisy surface with dead points, plus a
    second slot's partial layer inside the radius) against its definition solved
    another way: for each point, the weighted least-squares algebraic sphere
    s = u0 + u1 x + u2 y + z + u4 (x^2 + y^2 + z^2) over the alive points of every
    slot in the window (local coordinates over h, weight (1 - d^2)^4 inside the
    unit ball) by numpy's lstsq on the square-root-weighted design, and the
    point moved along the line of sight to the root of s(0, 0, z) nearest to it
    (numpy's polynomial roots), within one radius and the histogram."""
    rng = np.random.default_rng(21)
    h, w, t = 13, 15, 2000
    prm = _params(k_max=2)
    pitch, hh, R = prm["pixel_pitch"], prm["apss_radius"], prm["win_r"]
    i, j = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    front = 700 + 4.0 * j - 2.5 * i + 0.35 * (i - 6) ** 2 - 0.2 * (j - 7) * (i - 6) + rng.normal(0, 2.5, (h, w))
    front[rng.random((h, w)) < 0.15] = np.inf                       # dead points
    layer = front + 25.0 + rng.normal(0, 2.0, (h, w))
    layer[rng.random((h, w)) < 0.7] = np.inf
    st = _cloud(orc, np.stack([front, layer]))
    src_t, src_a = st.t.copy(), st.alive.copy()
    orc.apss(h, w, t, prm, st)
    checked = skipped = 0
    for k in range(2):
        for a in range(h):
            for b in range(w):
                if not src_a[k, a, b]:
                    continue
                t0 = src_t[k, a, b]
                rows, wts, offs = [], [], []
                for m in range(2):
                    for di in range(-R, R + 1):
                        for dj in range(-R, R + 1):
                            ii, jj = a + di, b + dj
                            if not (0 <= ii < h and 0 <= jj < w) or not src_a[m, ii, jj]:
                                continue
                            x, y, z = pitch * dj / hh, pitch * di / hh, (src_t[m, ii, jj] - t0) / hh
                            d2 = x * x + y * y + z * z
                            if d2 < 1.0:
                                rows.append((x, y, z, d2))
                                wts.append((1.0 - d2) ** 4)
                                offs.append((di, dj))
                got = st.t[k, a, b]
                o = np.array(offs, np.float64).reshape(-1, 2)
                if len(rows) < prm["apss_min_nb"] or np.linalg.matrix_rank(np.c_[np.ones(len(o)), o]) < 3:
                    assert got == t0
                    continue
                r = np.array(rows)
                sw = np.sqrt(np.array(wts))
                A = np.c_[np.ones(len(r)), r[:, 0], r[:, 1], r[:, 3]] * sw[:, None]
                u0, _, _, u4 = np.linalg.lstsq(A, -r[:, 2] * sw, rcond=None)[0]
                roots = np.roots([u4, 1.0, u0]) if abs(u4) > 1e-12 else np.array([-u0])
                real = roots[np.abs(roots.imag) < 1e-12].real
                if len(real) == 0:
                    skipped += 1
                    continue
                zs = float(np.clip(real[np.argmin(np.abs(real))], -1.0, 1.0))
                want = float(np.clip(t0 + hh * zs, 0.0, t - 1.0))
                assert abs(got - want) < 1e-7, (k, a, b, got, want)
                checked += 1
    assert checked > 150 and skipped <= 0.02 * checked


def test_intensity_lowpass_pruning_and_merge_on_a_generic_cloud(orc):
    """The intensity denoiser on a generic cloud (curved noisy front surface with
    dead points, a second slot's partial layer inside the radius, random
    intensities) against its definition evaluated by brute force: each alive
    point's intensity becomes the (1 - d^2/h^2)^4-weighted mean of the
    intensities of the alive points of every slot in its window within the 3-D
    radius (itself included), points below r_min are removed, and two alive
    points of one pixel closer in depth than merge_dist become one: the weaker
    (the later slot on a tie) is removed and its intensity added to the other."""
    rng = np.random.default_rng(33)
    h, w = 11, 14
    prm = _params(k_max=2, r_min=2.2, merge_dist=12.0)
    pitch, hr, R = prm["pixel_pitch"], prm["int_radius"], prm["win_r"]
    i, j = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    front = 600 + 3.0 * j - 2.0 * i + 0.3 * (i - 5) ** 2 + rng.normal(0, 2.5, (h, w))
    front[rng.random((h, w)) < 0.15] = np.inf
    layer = front + rng.uniform(5.0, 30.0, (h, w))
    layer[rng.random((h, w)) < 0.6] = np.inf
    st = _cloud(orc, np.stack([front, layer]))
    st.r[:] = rng.uniform(0.5, 5.0, st.r.shape)
    t0, r0, a0 = st.t.copy(), st.r.copy(), st.alive.copy()
    orc.int_lowpass(h, w, prm, st)
    rbar = r0.copy()
    for k in range(2):
        for a in range(h):
            for b in range(w):
                if not a0[k, a, b]:
                    continue
                num = den = 0.0
                for m in range(2):
                    for ii in range(max(0, a - R), min(h, a + R + 1)):
                        for jj in range(max(0, b - R), min(w, b + R + 1)):
                            if not a0[m, ii, jj]:
                                continue
                            d2 = ((pitch * (jj - b)) ** 2 + (pitch * (ii - a)) ** 2
                                  + (t0[m, ii, jj] - t0[k, a, b]) ** 2) / hr ** 2
                            if d2 < 1.0:
                                num += (1.0 - d2) ** 4 * r0[m, ii, jj]
                                den += (1.0 - d2) ** 4
                rbar[k, a, b] = num / den
    alive = a0.astype(bool) & (rbar.astype(np.float32) >= np.float32(prm["r_min"]))
    want = rbar.copy()
    merged = 0
    for a in range(h):
        for b in range(w):
            if alive[0, a, b] and alive[1, a, b] and abs(t0[0, a, b] - t0[1, a, b]) < prm["merge_dist"]:
                keep, drop = (1, 0) if want[1, a, b] > want[0, a, b] else (0, 1)
                want[keep, a, b] += want[drop, a, b]
                alive[drop, a, b] = False
                merged += 1
    assert merged > 3 and (a0.astype(bool) & ~alive).sum() > merged      # both rules were exercised
    assert np.array_equal(st.alive.astype(bool), alive)
    on = alive
    np.testing.assert_allclose(st.r[on], want[on], rtol=1e-12)
    # an exact tie (no low-pass): the later slot is the one removed
    tie = _cloud(orc, np.array([[[100.0]], [[105.0]]]))
    tie.r[:] = 3.0
    orc.int_lowpass(1, 1, _params(k_max=2, r_min=0.5, merge_dist=12.0, intensity_denoiser=0), tie)
    assert tie.alive[:, 0, 0].tolist() == [1, 0] and tie.r[0, 0, 0] == 6.0


def _generic_two_slot_cloud(orc, seed, h=13, w=15):
    """A curved, noisy front surface with dead points plus a second slot's
    partial layer inside the radius (the generic cloud of the lstsq pins)."""
    rng = np.random.default_rng(seed)
    i, j = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    front = 700 + 4.0 * j - 2.5 * i + 0.35 * (i - 6) ** 2 - 0.2 * (j - 7) * (i - 6) + rng.normal(0, 2.5, (h, w))
    front[rng.random((h, w)) < 0.15] = np.inf
    layer = front + 25.0 + rng.normal(0, 2.0, (h, w))
    layer[rng.random((h, w)) < 0.7] = np.inf
    return _cloud(orc, np.stack([front, layer]))


def _window(src_t, src_a, k, a, b, prm, h, w):
    """Neighbours of point (k, a, b) by their definition: (x, y, z, d2, weight, di, dj)."""
    pitch, hh, R = prm["pixel_pitch"], prm["apss_radius"], prm["win_r"]
    t0 = src_t[k, a, b]
    out = []
    for m in range(src_t.shape[0]):
        for di in range(-R, R + 1):
            for dj in range(-R, R + 1):
                ii, jj = a + di, b + dj
                if not (0 <= ii < h and 0 <= jj < w) or not src_a[m, ii, jj]:
                    continue
                x, y, z = pitch * dj / hh, pitch * di / hh, (src_t[m, ii, jj] - t0) / hh
                d2 = x * x + y * y + z * z
                if d2 < 1.0:
                    out.append((x, y, z, d2, (1.0 - d2) ** 4, di, dj))
    return np.array(out, np.float64).reshape(-1, 7)


def test_plane_fit_matches_weighted_least_squares_plane_by_lstsq(orc):
    """The plane-fit depth denoiser on a generic cloud against its definition
    solved another way: the weighted least-squares plane u0 + u1 x + u2 y = -z
    over the window's weighted neighbours by numpy's lstsq on the
    square-root-weighted design, the point moved to z* = -u0 (within one
    radius and the histogram); points with too few neighbours or collinear
    pixel offsets stay."""
    h, w, t = 13, 15, 2000
    prm = _params(k_max=2)
    st = _generic_two_slot_cloud(orc, 22, h, w)
    src_t, src_a = st.t.copy(), st.alive.copy()
    orc.plane(h, w, t, prm, st)
    checked = 0
    for k in range(2):
        for a in range(h):
            for b in range(w):
                if not src_a[k, a, b]:
                    continue
                nb = _window(src_t, src_a, k, a, b, prm, h, w)
                got, t0 = st.t[k, a, b], src_t[k, a, b]
                if len(nb) < prm["apss_min_nb"] or np.linalg.matrix_rank(np.c_[np.ones(len(nb)), nb[:, 5:7]]) < 3:
                    assert got == t0
                    continue
                sw = np.sqrt(nb[:, 4])
                A = np.c_[np.ones(len(nb)), nb[:, 0], nb[:, 1]] * sw[:, None]
                u0 = np.linalg.lstsq(A, -nb[:, 2] * sw, rcond=None)[0][0]
                want = float(np.clip(t0 + prm["apss_radius"] * np.clip(-u0, -1, 1), 0, t - 1))
                assert abs(got - want) < 1e-7, (k, a, b, got, want)
                checked += 1
    assert checked > 150


def test_plane_fit_keeps_planes_but_not_spheres(orc):
    """Exact planes are fixed points of the plane fit (as of APSS); an exact
    sphere, which APSS keeps, is flattened: the sphere term is what the plane
    fit drops."""
    h, w = 15, 15
    prm = _params(pixel_pitch=4.0, apss_radius=12.0)
    i, j = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    plane = 500.0 + 1.3 * 4.0 * i - 0.6 * 4.0 * j
    st = _cloud(orc, plane)
    orc.plane(h, w, 2000, prm, st)
    np.testing.assert_allclose(st.t[0], plane, atol=1e-9)
    x, y = 4.0 * (j - 7.2), 4.0 * (i - 6.9)
    sphere = 900.0 - np.sqrt(60.0 ** 2 - x ** 2 - y ** 2)
    a, b = _cloud(orc, sphere), _cloud(orc, sphere)
    orc.apss(h, w, 2000, prm, a)
    orc.plane(h, w, 2000, prm, b)
    np.testing.assert_allclose(a.t[0], sphere, atol=1e-9)
    assert np.abs(b.t[0] - sphere)[3:-3, 3:-3].min() > 1e-3


def test_bilateral_matches_weighted_mean_by_brute_force(orc):
    """The bilateral depth denoiser on a generic cloud against its definition:
    the point's depth offset becomes the weight-averaged offset of the
    window's weighted neighbours (itself included); it commutes with a depth
    shift and keeps a fronto-parallel plane."""
    h, w, t = 13, 15, 2000
    prm = _params(k_max=2)
    st = _generic_two_slot_cloud(orc, 23, h, w)
    src_t, src_a = st.t.copy(), st.alive.copy()
    orc.bilateral(h, w, t, prm, st)
    checked = 0
    for k in range(2):
        for a in range(h):
            for b in range(w):
                if not src_a[k, a, b]:
                    continue
                nb = _window(src_t, src_a, k, a, b, prm, h, w)
                got, t0 = st.t[k, a, b], src_t[k, a, b]
                if len(nb) < prm["apss_min_nb"]:
                    assert got == t0
                    continue
                zs = float((nb[:, 4] * nb[:, 2]).sum() / nb[:, 4].sum())
                want = float(np.clip(t0 + prm["apss_radius"] * zs, 0, t - 1))
                assert abs(got - want) < 1e-7, (k, a, b, got, want)
                checked += 1
    assert checked > 150
    shifted = _generic_two_slot_cloud(orc, 23, h, w)
    shifted.t[:] = src_t + 37.5
    orc.bilateral(h, w, t, prm, shifted)
    np.testing.assert_allclose(shifted.t - 37.5, st.t, atol=1e-9)
    flat = _cloud(orc, np.full((9, 9), 812.25))
    orc.bilateral(9, 9, t, prm, flat)
    assert np.all(flat.t[0] == 812.25)
