"""Pins of the oracle's observation model, gradients and gradient steps."""
import numpy as np
import pytest
from scipy import optimize

import scenes


def _irf(orc, sigma=2.5, half=10):
    g = scenes.gaussian_irf(sigma, half)
    return orc.OIrf(g.samples, g.origin)


def _params(**over):
    sc = scenes.small_random(4, 4, 64)
    p = scenes.make_params(sc)
    p.update(over)
    return p


def test_irf_interpolates_samples_and_partition_of_unity(orc):
    g = scenes.gamma_irf(3, 5, 40)
    irf = orc.OIrf(g.samples, g.origin)
    for k in range(len(irf.h)):
        h, _ = orc.irf_eval(irf, k - irf.origin)
        assert abs(h - irf.h[k]) < 1e-15
    # cubic convolution reproduces constants: sum over bins of h(t - tau) = 1
    for tau in (50.0, 50.25, 63.7, 71.999):
        tot = sum(orc.irf_eval(irf, t - tau)[0] for t in range(0, 200))
        assert abs(tot - 1.0) < 1e-12
        dtot = sum(orc.irf_eval(irf, t - tau)[1] for t in range(0, 200))
        assert abs(dtot) < 1e-12


def test_irf_derivative_matches_finite_difference(orc):
    irf = _irf(orc)
    for x in np.linspace(-11.7, 11.7, 37):
        if abs(x - round(x)) < 1e-3:
            continue
        eps = 1e-6
        hp, _ = orc.irf_eval(irf, x + eps)
        hm, _ = orc.irf_eval(irf, x - eps)
        _, dh = orc.irf_eval(irf, x)
        assert abs((hp - hm) / (2 * eps) - dh) < 1e-7


def _random_state(orc, rng, k, h, w, t, edge=False):
    st = orc.new_state(k, h, w)
    st.t[:] = rng.uniform(15, t - 15, size=(k, h, w))
    if edge:
        st.t[0, 0, 0] = 1.3
        st.t[-1, -1, -1] = t - 2.4
    st.r[:] = rng.uniform(0.5, 6.0, size=(k, h, w))
    st.alive[:] = (rng.random((k, h, w)) < 0.8).astype(np.uint8)
    st.b[:] = rng.uniform(0.01, 0.2, size=(h, w))
    return st


@pytest.mark.parametrize("edge", [False, True])
def test_sparse_gradients_match_finite_differences(orc, edge):
    """dg/dt, dg/dr, dg/db from the nonzero-bin form equal central differences of
    the dense negative log-likelihood (Results, "Observation model")."""
    rng = np.random.default_rng(1 if edge else 2)
    k, h, w, t = 2, 2, 3, 64
    irf = _irf(orc)
    st = _random_state(orc, rng, k, h, w, t, edge)
    z = rng.poisson(0.6, size=(h, w, t)).astype(np.float64)
    gain = rng.uniform(0.5, 1.5, size=(h, w))
    prm = _params(k_max=k)
    fr = orc.OFrame(z, gain)
    gt, gr, gb = orc.gradients(fr, st, irf, prm)

    def f(s):
        return orc.nll_dense(z, gain, s, irf, prm["lam_floor"])

    for kk in range(k):
        for i in range(h):
            for j in range(w):
                if not st.alive[kk, i, j]:
                    assert gt[kk, i, j] == 0 and gr[kk, i, j] == 0
                    continue
                for arr, grad, eps in ((st.t, gt, 1e-5), (st.r, gr, 1e-6)):
                    sp, sm = st.copy(), st.copy()
                    getattr(sp, "t" if arr is st.t else "r")[kk, i, j] += eps
                    getattr(sm, "t" if arr is st.t else "r")[kk, i, j] -= eps
                    fd = (f(sp) - f(sm)) / (2 * eps)
                    assert abs(fd - grad[kk, i, j]) < 2e-6 * max(1.0, abs(fd)), (kk, i, j, fd, grad[kk, i, j])
    for i in range(h):
        for j in range(w):
            sp, sm = st.copy(), st.copy()
            sp.b[i, j] += 1e-7
            sm.b[i, j] -= 1e-7
            fd = (f(sp) - f(sm)) / 2e-7
            assert abs(fd - gb[i, j]) < 2e-5 * max(1.0, abs(fd))


def _expected_counts(orc, irf, st, t, gain=None):
    """lambda of the likelihood equation, written out bin by bin."""
    k, h, w = st.t.shape
    lam = np.zeros((h, w, t))
    for i in range(h):
        for j in range(w):
            g = 1.0 if gain is None else gain[i, j]
            for tb in range(t):
                acc = st.b[i, j]
                for kk in range(k):
                    if st.alive[kk, i, j]:
                        acc += st.r[kk, i, j] * orc.irf_eval(irf, tb - st.t[kk, i, j])[0]
                lam[i, j, tb] = g * acc
    return lam


def test_gradient_vanishes_at_truth_with_expected_counts(orc):
    """With z = lambda(truth) every term 1 - z/lambda vanishes, so all gradients
    are zero, for points deep inside and at the edges of the histogram.  (The
    background stays positive: the cubic interpolant has a small negative lobe
    beyond the IRF support, where a zero background would give lambda < 0.)"""
    rng = np.random.default_rng(5)
    irf = _irf(orc)
    for bkg in (0.05, 1e-3):
        st = _random_state(orc, rng, 2, 2, 2, 48, edge=True)
        st.alive[:] = 1
        st.b[:] = bkg
        z = _expected_counts(orc, irf, st, 48)
        fr = orc.OFrame(z)
        gt, gr, gb = orc.gradients(fr, st, irf, _params(k_max=2))
        assert np.abs(gt).max() < 1e-10
        assert np.abs(gr).max() < 1e-10
        assert np.abs(gb).max() < 1e-9


def test_noise_free_recovery_without_denoisers(orc):
    """Gradient steps alone, fed the expected counts of a known cloud, return
    that cloud from a perturbed start."""
    rng = np.random.default_rng(7)
    irf = _irf(orc)
    k, h, w, t = 2, 2, 2, 96
    truth = orc.new_state(k, h, w)
    truth.t[0] = rng.uniform(20, 35, (h, w))
    truth.t[1] = rng.uniform(55, 75, (h, w))
    truth.r[:] = rng.uniform(20, 60, (k, h, w))
    truth.alive[:] = 1
    truth.b[:] = rng.uniform(0.05, 0.2, (h, w))
    z = _expected_counts(orc, irf, truth, t)
    fr = orc.OFrame(z)
    st = truth.copy()
    st.t += rng.uniform(-1.5, 1.5, st.t.shape)
    st.r *= rng.uniform(0.7, 1.3, st.r.shape)
    st.b *= 1.5
    prm = _params(k_max=k, depth_denoiser=0, intensity_denoiser=0, r_min=1e-3)
    orc.palm(fr, irf, prm, st, 400)
    np.testing.assert_allclose(st.t, truth.t, atol=1e-6)
    np.testing.assert_allclose(st.r, truth.r, rtol=1e-6)
    np.testing.assert_allclose(st.b, truth.b, rtol=1e-5)


def test_single_pixel_matches_brute_force_mle(orc):
    """One pixel, one surface, no denoiser: the loop converges to the maximum-
    likelihood depth, found here by a 1e-3-bin grid over t with (r, b) profiled
    out by a generic bounded optimiser."""
    rng = np.random.default_rng(11)
    irf = _irf(orc, sigma=3.0, half=12)
    t = 80
    truth = orc.new_state(1, 1, 1)
    truth.t[:] = 37.3
    truth.r[:] = 30.0
    truth.alive[:] = 1
    truth.b[:] = 0.05
    lam = _expected_counts(orc, irf, truth, t)
    z = rng.poisson(lam).astype(np.float64)
    fr = orc.OFrame(z)
    st = truth.copy()
    st.t[:] = 36.0
    st.r[:] = 20.0
    st.b[:] = 0.1
    prm = _params(k_max=1, depth_denoiser=0, intensity_denoiser=0, r_min=1e-3)
    orc.palm(fr, irf, prm, st, 600)

    hvals = {}

    def prof(tt):
        hv = np.array([orc.irf_eval(irf, tb - tt)[0] for tb in range(t)])
        hvals[tt] = hv

        def nll(v):
            r, b = v
            lam_ = np.maximum(r * hv + b, 1e-9)
            return float(np.sum(lam_ - z[0, 0] * np.log(lam_)))
        res = optimize.minimize(nll, x0=[20.0, 0.1], bounds=[(1e-6, None), (1e-8, None)],
                                method="L-BFGS-B", options=dict(ftol=1e-15, gtol=1e-12))
        return res.fun
    coarse = np.arange(33.0, 41.0, 0.05)
    c0 = coarse[int(np.argmin([prof(x) for x in coarse]))]
    fine = np.arange(c0 - 0.06, c0 + 0.06, 1e-3)
    best = fine[int(np.argmin([prof(x) for x in fine]))]
    assert abs(st.t[0, 0, 0] - best) < 2e-3, (st.t[0, 0, 0], best)


def test_step_projections(orc):
    """Intensities stay >= 0, backgrounds >= b_floor, depths inside [0, T-1] and
    each depth move is at most dt_max."""
    rng = np.random.default_rng(3)
    irf = _irf(orc)
    st = _random_state(orc, rng, 2, 3, 3, 64, edge=True)
    z = rng.poisson(3.0, size=(3, 3, 64)).astype(np.float64)
    fr = orc.OFrame(z)
    prm = _params(k_max=2, dt_max=0.75)
    before = st.t.copy()
    orc.t_step(fr, irf, prm, st)
    assert np.all(np.abs(st.t - before) <= 0.75 + 1e-12)
    assert st.t.min() >= 0 and st.t.max() <= 63
    orc.r_step(fr, irf, prm, st)
    assert st.r.min() >= 0
    st.b[:] = 0.0
    z2 = np.zeros_like(z)
    orc.b_step(orc.OFrame(z2), irf, prm, st)
    assert st.b.min() >= np.float32(prm["b_floor"])


def test_unit_steps_are_em_updates_and_never_raise_the_nll(orc):
    """With step 1 and no regulariser offsets, the intensity and background steps
    are the EM (Richardson-Lucy) updates of the Poisson mixture: each slot's
    intensity is multiplied by its share of the photons, sum z h_k/lambda over
    sum h_k, and the background by sum z/lambda over T, all slots of a pixel
    from the same lambda.  EM never raises the negative log-likelihood, so
    alternating the two steps gives a non-increasing NLL."""
    rng = np.random.default_rng(8)
    irf = _irf(orc)
    t = 120
    st = orc.new_state(2, 1, 2)
    st.t[:, 0, :] = [[30.4, 47.9], [82.25, 71.6]]
    st.r[:] = rng.uniform(2.0, 9.0, st.r.shape)
    st.alive[:] = 1
    st.b[:] = [[0.15, 0.4]]
    z = rng.poisson(2.0, size=(1, 2, t)).astype(np.float64)
    prm = _params(k_max=2, r_step=1.0, eps_r=0.0, b_step=1.0, eps_b=0.0)
    fr = orc.OFrame(z)

    def em(s):
        r, b = s.r.copy(), s.b.copy()
        for p in range(2):
            hk = np.array([[orc.irf_eval(irf, tb - s.t[k, 0, p])[0] for tb in range(t)] for k in range(2)])
            lam = b[0, p] + r[:, 0, p] @ hk
            r[:, 0, p] = s.r[:, 0, p] * (hk @ (z[0, p] / lam)) / hk.sum(axis=1)
            b[0, p] = s.b[0, p] * np.sum(z[0, p] / lam) / t
        return r, b

    want_r, _ = em(st)
    orc.r_step(fr, irf, prm, st)
    np.testing.assert_allclose(st.r, want_r, rtol=1e-12)
    _, want_b = em(st)
    orc.b_step(fr, irf, prm, st)
    np.testing.assert_allclose(st.b, want_b, rtol=1e-12)
    nll = [orc.nll_dense(z, None, st, irf, prm["lam_floor"])]
    for _ in range(60):
        orc.r_step(fr, irf, prm, st)
        orc.b_step(fr, irf, prm, st)
        nll.append(orc.nll_dense(z, None, st, irf, prm["lam_floor"]))
    assert all(b <= a + 1e-9 * abs(a) for a, b in zip(nll, nll[1:]))
    assert nll[-1] < nll[0]


@pytest.mark.parametrize("tstar,delta", [(50.3, 0.02), (50.3, -0.03), (3.4, 0.02), (96.1, -0.02)])
def test_depth_step_is_a_half_fisher_scoring_step(orc, tstar, delta):
    """With noise-free counts and t_step = (g r / F) / 2, F = sum (g r h')^2 / lambda
    the Fisher information of the depth at the truth, the depth step is half a
    Fisher-scoring step: a small error delta becomes delta / 2 to first order,
    from either side, also where the histogram's ends cut the IRF's support
    (there the derivative of the IRF mass inside the histogram enters the
    gradient)."""
    irf = _irf(orc)
    t, r, b = 100, 500.0, 0.05
    hv = np.array([orc.irf_eval(irf, tb - tstar) for tb in range(t)])
    lam = b + r * hv[:, 0]
    fisher = np.sum((r * hv[:, 1]) ** 2 / lam)
    st = orc.new_state(1, 1, 1)
    st.t[:] = tstar + delta
    st.r[:] = r
    st.b[:] = b
    st.alive[:] = 1
    prm = _params(k_max=1, t_step=0.5 * r / fisher, eps_r=0.0, lam_floor=1e-12)
    orc.t_step(orc.OFrame(lam.reshape(1, 1, t)), irf, prm, st)
    ratio = (st.t[0, 0, 0] - tstar) / delta
    assert abs(ratio - 0.5) < 0.03, ratio
