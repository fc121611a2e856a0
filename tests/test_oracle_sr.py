"""Pins of the oracle's super-resolution: the point-to-cube mapping f of
Results, "Observation model" sending a u x u window of world pixels to one
lidar pixel (Results, "3D Dynamic scenes")."""
import numpy as np

import scenes


def _irf(orc):
    g = scenes.gaussian_irf(1.5, 6)
    return orc.OIrf(g.samples, g.origin)


def _params(**over):
    p = scenes.make_params(scenes.small_random(4, 4, 64))
    p.update(dict(pixel_pitch=4.0, apss_radius=14.0, int_radius=14.0, upsample=3))
    p.update(over)
    return p


def _lambda_sr(orc, irf, st, h, w, t, up, gain=None):
    """lambda of every lidar pixel and bin, summing the alive points of its
    u x u world pixels, written out point by point."""
    lam = np.zeros((h, w, t))
    k = st.t.shape[0]
    for i in range(h):
        for j in range(w):
            g = 1.0 if gain is None else gain[i, j]
            for tb in range(t):
                acc = st.b[i, j]
                for a in range(up):
                    for c in range(up):
                        for kk in range(k):
                            if st.alive[kk, up * i + a, up * j + c]:
                                acc += st.r[kk, up * i + a, up * j + c] * \
                                    orc.irf_eval(irf, tb - st.t[kk, up * i + a, up * j + c])[0]
                lam[i, j, tb] = g * acc
    return lam


def test_super_resolved_gradients_match_finite_differences(orc):
    """Per world point dg/dt and dg/dr, per lidar pixel dg/db, against central
    differences of the dense negative log-likelihood whose lambda sums each
    lidar pixel's u x u block; the NLL equals sum(lambda - z log lambda) over
    the block sums written out point by point."""
    rng = np.random.default_rng(5)
    up, k, h, w, t = 3, 2, 2, 2, 40
    irf = _irf(orc)
    st = orc.new_state(k, h, w, up)
    st.t[:] = rng.uniform(4, t - 4, size=st.t.shape)
    st.t[0, 0, 0] = 1.2
    st.r[:] = rng.uniform(0.2, 2.0, size=st.r.shape)
    st.alive[:] = (rng.random(st.alive.shape) < 0.8).astype(np.uint8)
    st.b[:] = rng.uniform(0.02, 0.2, size=(h, w))
    z = rng.poisson(1.5, size=(h, w, t)).astype(np.float64)
    gain = rng.uniform(0.5, 1.5, size=(h, w))
    prm = _params(k_max=k)
    fr = orc.OFrame(z, gain)
    gt, gr, gb = orc.gradients(fr, st, irf, prm)

    def f(s):
        return orc.nll_dense(z, gain, s, irf, prm["lam_floor"], up=up)

    lam = _lambda_sr(orc, irf, st, h, w, t, up, gain)
    assert abs(f(st) - (lam - z * np.log(lam)).sum()) < 1e-9 * abs(f(st))
    for kk in range(k):
        for i in range(h * up):
            for j in range(w * up):
                if not st.alive[kk, i, j]:
                    assert gt[kk, i, j] == 0 and gr[kk, i, j] == 0
                    continue
                for name, grad, eps in (("t", gt, 1e-5), ("r", gr, 1e-6)):
                    sp, sm = st.copy(), st.copy()
                    getattr(sp, name)[kk, i, j] += eps
                    getattr(sm, name)[kk, i, j] -= eps
                    fd = (f(sp) - f(sm)) / (2 * eps)
                    assert abs(fd - grad[kk, i, j]) < 2e-6 * max(1.0, abs(fd)), (name, kk, i, j)
    for i in range(h):
        for j in range(w):
            sp, sm = st.copy(), st.copy()
            sp.b[i, j] += 1e-7
            sm.b[i, j] -= 1e-7
            assert abs((f(sp) - f(sm)) / 2e-7 - gb[i, j]) < 2e-5 * max(1.0, abs(gb[i, j]))


def test_noise_free_world_plane_is_a_fixed_point(orc):
    """Noise-free counts of a slanted plane at world resolution (12 x 15 world
    pixels seen through 4 x 5 lidar pixels, u = 3), the state started at the
    truth: the whole super-resolved iteration (gradient steps, APSS on the
    world grid, intensity low-pass, background step) leaves it in place."""
    up, h, w, t = 3, 4, 5, 120
    irf = _irf(orc)
    prm = _params(k_max=1, n_iter=4, bkg_mode=0)
    st = orc.new_state(1, h, w, up)
    ii, jj = np.meshgrid(np.arange(h * up), np.arange(w * up), indexing="ij")
    st.t[0] = 50.0 + 0.35 * 4.0 * ii - 0.2 * 4.0 * jj
    st.r[0] = 2.0
    st.alive[:] = 1
    st.b[:] = 0.05
    z = _lambda_sr(orc, irf, st, h, w, t, up)
    fr = orc.OFrame(z)
    out = st.copy()
    orc.palm(fr, irf, prm, out, prm["n_iter"])
    np.testing.assert_allclose(out.t, st.t, atol=1e-9)
    np.testing.assert_allclose(out.r, st.r, atol=1e-9)
    np.testing.assert_allclose(out.b, st.b, atol=1e-12)
    assert np.array_equal(out.alive, st.alive)


def test_block_permutation_invariance(orc):
    """lambda sees a lidar pixel's block as a set of points: exchanging two
    world pixels of one block leaves the NLL unchanged and exchanges their
    gradients."""
    rng = np.random.default_rng(6)
    up, k, h, w, t = 3, 2, 2, 3, 48
    irf = _irf(orc)
    st = orc.new_state(k, h, w, up)
    st.t[:] = rng.uniform(5, t - 5, size=st.t.shape)
    st.r[:] = rng.uniform(0.2, 2.0, size=st.r.shape)
    st.alive[:] = 1
    st.b[:] = 0.1
    z = rng.poisson(1.0, size=(h, w, t)).astype(np.float64)
    prm = _params(k_max=k)
    fr = orc.OFrame(z)
    g1 = orc.gradients(fr, st, irf, prm)
    sw = st.copy()
    for arr in (sw.t, sw.r, sw.alive):
        arr[:, 3, 4], arr[:, 5, 3] = arr[:, 5, 3].copy(), arr[:, 3, 4].copy()   # both in block (1, 1)
    g2 = orc.gradients(fr, sw, irf, prm)
    assert abs(orc.nll_dense(z, None, st, irf, 1e-9, up=up) - orc.nll_dense(z, None, sw, irf, 1e-9, up=up)) < 1e-9
    for a, b in zip(g1[:2], g2[:2]):
        np.testing.assert_allclose(a[:, 3, 4], b[:, 5, 3], rtol=1e-12)
        np.testing.assert_allclose(a[:, 5, 3], b[:, 3, 4], rtol=1e-12)
    np.testing.assert_allclose(g1[2], g2[2], rtol=1e-12)


def test_super_resolved_init_spreads_each_pixels_peaks_over_its_block(orc):
    """The initialisation gives every world pixel of a lidar pixel's block
    that pixel's peaks with 1/u^2 of the intensity (so the block's lambda is
    the pixel's), and the same background."""
    sc = scenes.small_random(5, 6, 200, n_comp=2, seed=7)
    z = orc.synthesize(scenes.sampling_tables(sc))
    irf = orc.OIrf(sc.irf.samples, sc.irf.origin)
    prm = scenes.make_params(sc)
    a = orc.init(z, None, irf, prm)
    b = orc.init(z, None, irf, dict(prm, upsample=3))
    assert b.t.shape == (prm["k_max"], 15, 18) and b.b.shape == (5, 6)
    rep = lambda x: np.repeat(np.repeat(x, 3, axis=1), 3, axis=2)
    assert np.array_equal(b.t, rep(a.t))
    assert np.array_equal(b.alive, rep(a.alive))
    np.testing.assert_allclose(b.r, rep(a.r) / 9.0, rtol=1e-15)
    assert np.array_equal(b.b, a.b)
