"""Pins of the oracle's whole reconstruction (initialisation + PALM loop with the
denoisers), which the paper gives no worked example for: convergence to a
known cloud from noise-free data, and the symmetries the method has -- the
histogram's time axis (a shift of every photon shifts every depth) and the
pixel grid (a transposed or mirrored frame gives the transposed or mirrored
cloud).  A dropped or misplaced term, a wrong index into the bins or a
swapped window axis breaks one of them."""
import numpy as np
import pytest

import scenes


def _irf(orc, sigma=2.5, half=10):
    g = scenes.gaussian_irf(sigma, half)
    return orc.OIrf(g.samples, g.origin)


def _expected_counts(orc, irf, st, t):
    """lambda of the likelihood equation, bin by bin (gain 1)."""
    k, h, w = st.t.shape
    lam = np.zeros((h, w, t))
    for i in range(h):
        for j in range(w):
            for tb in range(t):
                acc = st.b[i, j]
                for kk in range(k):
                    if st.alive[kk, i, j]:
                        acc += st.r[kk, i, j] * orc.irf_eval(irf, tb - st.t[kk, i, j])[0]
                lam[i, j, tb] = acc
    return lam


def test_loop_with_denoisers_recovers_two_slanted_planes(orc):
    """Noise-free counts of two slanted planes (different slopes along the two
    image axes, a constant intensity each): the truth is a fixed point of every
    step (zero gradients, APSS keeps planes, the low-pass keeps constants), and
    the full loop with APSS and the intensity low-pass returns it from a
    perturbed start."""
    rng = np.random.default_rng(5)
    irf = _irf(orc)
    k, h, w, t = 2, 9, 11, 128
    i, j = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    truth = orc.new_state(k, h, w)
    truth.t[0] = 30.0 + 0.45 * j + 0.15 * i
    truth.t[1] = 85.0 + 0.10 * j - 0.35 * i
    truth.r[0] = 40.0
    truth.r[1] = 25.0
    truth.alive[:] = 1
    truth.b[:] = 0.1
    z = _expected_counts(orc, irf, truth, t)
    prm = scenes.make_params(scenes.small_random(4, 4, 64), k_max=k, pixel_pitch=4.0, apss_radius=12.0,
                             int_radius=12.0, win_r=3, r_min=1e-3, merge_dist=5.0, depth_denoiser=1,
                             intensity_denoiser=1, bkg_mode=0)
    st = truth.copy()
    orc.palm(orc.OFrame(z), irf, prm, st, 3)
    # the truth is a fixed point of the whole iteration
    np.testing.assert_allclose(st.t, truth.t, atol=1e-9)
    np.testing.assert_allclose(st.r, truth.r, rtol=1e-9)
    np.testing.assert_allclose(st.b, truth.b, rtol=1e-7)
    # and the loop returns to it from a perturbed start
    st = truth.copy()
    st.t += rng.uniform(-1.0, 1.0, st.t.shape)
    st.r *= rng.uniform(0.8, 1.2, st.r.shape)
    st.b *= 1.5
    orc.palm(orc.OFrame(z), irf, prm, st, 300)
    assert st.alive.all()
    np.testing.assert_allclose(st.t, truth.t, atol=1e-4)
    np.testing.assert_allclose(st.r, truth.r, rtol=1e-4)
    np.testing.assert_allclose(st.b, truth.b, rtol=1e-3)


def _photon_frame(orc, h, w, t, seed):
    """Poisson counts of a smooth two-surface scene with no background photons
    (so nothing but the surfaces' returns sits in the histogram, all of them at
    least 28 bins from either end)."""
    sc = scenes.small_random(h, w, t, n_comp=2, seed=seed, bkg=0.0)
    z = orc.synthesize(scenes.sampling_tables(sc))
    irf = orc.OIrf(sc.irf.samples, sc.irf.origin)
    return sc, z, irf


def _assert_same_cloud(a, b, dt=0.0):
    assert np.array_equal(a.alive, b.alive)
    on = a.alive.astype(bool)
    np.testing.assert_allclose(b.t[on], a.t[on] + dt, atol=1e-9)
    np.testing.assert_allclose(b.r[on], a.r[on], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(b.b, a.b, rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("shift", [1, 17])
def test_reconstruction_is_shift_equivariant_in_time(orc, shift):
    sc, z, irf = _photon_frame(orc, 8, 10, 192, seed=3)
    assert not z[..., -(shift + 1):].any()
    zs = np.zeros_like(z)
    zs[..., shift:] = z[..., :-shift]
    prm = scenes.make_params(sc, n_iter=8)
    a = orc.reconstruct(z, irf, prm)
    b = orc.reconstruct(zs, irf, prm)
    assert a.alive.sum() > 0
    _assert_same_cloud(a, b, dt=float(shift))


def test_reconstruction_is_equivariant_under_transposition_and_mirroring(orc):
    sc, z, irf = _photon_frame(orc, 7, 11, 160, seed=9)
    prm = scenes.make_params(sc, n_iter=8)
    a = orc.reconstruct(z, irf, prm)
    assert a.alive.sum() > 0
    tr = orc.reconstruct(np.ascontiguousarray(z.transpose(1, 0, 2)), irf, prm)
    ref = a.copy()
    ref.t = np.ascontiguousarray(a.t.transpose(0, 2, 1))
    ref.r = np.ascontiguousarray(a.r.transpose(0, 2, 1))
    ref.alive = np.ascontiguousarray(a.alive.transpose(0, 2, 1))
    ref.b = np.ascontiguousarray(a.b.T)
    _assert_same_cloud(ref, tr)
    mi = orc.reconstruct(np.ascontiguousarray(z[:, ::-1, :]), irf, prm)
    ref = a.copy()
    ref.t = np.ascontiguousarray(a.t[:, :, ::-1])
    ref.r = np.ascontiguousarray(a.r[:, :, ::-1])
    ref.alive = np.ascontiguousarray(a.alive[:, :, ::-1])
    ref.b = np.ascontiguousarray(a.b[:, ::-1])
    _assert_same_cloud(ref, mi)
