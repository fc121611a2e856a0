"""Pins of the oracle's per-pixel instrument responses: the likelihood of
Results, "Observation model" indexes the response h_{i,j} by pixel, so a
frame carries an index into a set of responses."""
import numpy as np
import pytest

import scenes


def _irfs(orc):
    a = scenes.gaussian_irf(2.5, 10)
    b = scenes.gamma_irf(3.0, 2.0, 30)
    return [orc.OIrf(a.samples, a.origin), orc.OIrf(b.samples, b.origin)]


def _params(**over):
    p = scenes.make_params(scenes.small_random(4, 4, 64))
    p.update(over)
    return p


def test_per_pixel_irf_gradients_match_finite_differences(orc):
    """dg/dt, dg/dr, dg/db with two responses mixed over the pixels equal
    central differences of the dense negative log-likelihood, itself the sum
    of the pixels' likelihoods each under its own response."""
    rng = np.random.default_rng(3)
    k, h, w, t = 2, 3, 3, 64
    irfs = _irfs(orc)
    idx = rng.integers(0, 2, size=(h, w)).astype(np.uint8)
    idx[0, 0], idx[0, 1] = 0, 1
    st = orc.new_state(k, h, w)
    st.t[:] = rng.uniform(3, t - 3, size=(k, h, w))
    st.t[0, 0, 1] = 1.7                         # response 1 cut by the histogram's start
    st.r[:] = rng.uniform(0.5, 6.0, size=(k, h, w))
    st.alive[:] = 1
    st.b[:] = rng.uniform(0.01, 0.2, size=(h, w))
    z = rng.poisson(0.6, size=(h, w, t)).astype(np.float64)
    gain = rng.uniform(0.5, 1.5, size=(h, w))
    prm = _params(k_max=k)
    fr = orc.OFrame(z, gain, irf_idx=idx)
    gt, gr, gb = orc.gradients(fr, st, irfs, prm)

    def f(s):
        return orc.nll_dense(z, gain, s, irfs, prm["lam_floor"], irf_idx=idx)

    total = 0.0
    for i in range(h):
        for j in range(w):
            one = orc.new_state(k, 1, 1)
            one.t[:, 0, 0], one.r[:, 0, 0] = st.t[:, i, j], st.r[:, i, j]
            one.alive[:, 0, 0], one.b[0, 0] = st.alive[:, i, j], st.b[i, j]
            total += orc.nll_dense(z[i:i + 1, j:j + 1], gain[i:i + 1, j:j + 1], one, irfs[idx[i, j]],
                                   prm["lam_floor"])
    assert abs(total - f(st)) < 1e-9 * abs(total)
    for kk in range(k):
        for i in range(h):
            for j in range(w):
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
            fd = (f(sp) - f(sm)) / 2e-7
            assert abs(fd - gb[i, j]) < 2e-5 * max(1.0, abs(fd))


def test_per_pixel_irfs_decouple_without_spatial_denoisers(orc):
    """Without the neighbourhood denoisers every pixel is reconstructed on its
    own, so a frame mixing two responses equals, pixel by pixel, the whole
    frame reconstructed under the response its index names (initialisation,
    matched filter, windows and all iterations included)."""
    sc = scenes.small_random(9, 11, 256, n_comp=2, seed=5)
    z = orc.synthesize(scenes.sampling_tables(sc))
    irfs = _irfs(orc)
    idx = (np.random.default_rng(4).random((sc.h, sc.w)) < 0.5).astype(np.uint8)
    prm = dict(scenes.make_params(sc), depth_denoiser=0, intensity_denoiser=0, bkg_mode=0, n_iter=8)
    mixed = orc.reconstruct(z, irfs, prm, irf_idx=idx)
    for i, irf in enumerate(irfs):
        alone = orc.reconstruct(z, irf, prm)
        m = idx == i
        for key in ("t", "r", "alive"):
            assert np.array_equal(getattr(mixed, key)[:, m], getattr(alone, key)[:, m]), (i, key)
        assert np.array_equal(mixed.b[m], alone.b[m])


@pytest.mark.parametrize("which", [0, 1])
def test_uniform_index_equals_the_single_response(orc, which):
    """Every pixel naming the same response is the single-response method."""
    sc = scenes.small_random(7, 8, 200, n_comp=2, seed=6)
    z = orc.synthesize(scenes.sampling_tables(sc))
    irfs = _irfs(orc)
    prm = scenes.make_params(sc)
    a = orc.reconstruct(z, irfs, prm, irf_idx=np.full((sc.h, sc.w), which, np.uint8))
    b = orc.reconstruct(z, irfs[which], prm)
    for key in ("t", "r", "alive", "b"):
        assert np.array_equal(getattr(a, key), getattr(b, key)), key
