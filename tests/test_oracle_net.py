"""Pins of the oracle's learned depth denoiser (an extension of the method that
stands in for the APSS depth step): each check rests on a fact the
mathematics fixes, not on the oracle's own formulas."""
import numpy as np
import pytest

import scenes
from oracle import oracle as O


def _rand_theta(rng, scale=0.2):
    th = np.zeros(O.net_nparams())
    for l, (ci, co) in enumerate(O.net_channels()):
        w0, b0, e = O.net_offset(l, False), O.net_offset(l, True), O.net_offset(l + 1, False)
        th[w0:b0] = rng.normal(0.0, scale / np.sqrt(9 * ci), b0 - w0)
        th[b0:e] = rng.normal(0.0, 0.05, e - b0)
    return th


def test_parameter_layout():
    ch = O.net_channels()
    assert ch == [(6, 48), (48, 48), (48, 48), (48, 2)]
    n = sum(co * ci * 9 + co for ci, co in ch)
    assert O.net_nparams() == n == 45074
    assert O.net_offset(0, False) == 0 and O.net_offset(0, True) == 48 * 6 * 9
    assert O.net_offset(3, True) + 2 == n


def test_bf16_rounding_is_nearest_even():
    # exact bfloat16 values stay, halfway cases go to the even mantissa
    assert list(O.bf16([1.0, -2.5, 0.0])) == [1.0, -2.5, 0.0]
    assert O.bf16([1 + 2 ** -8])[0] == 1.0                     # tie -> even (1.0)
    assert O.bf16([1 + 3 * 2 ** -8])[0] == 1 + 2 ** -6         # tie -> even (1.015625)
    rng = np.random.default_rng(0)
    x = rng.normal(0, 100, 2000)
    r = O.bf16(x)
    # the result has 8 significant bits and no bfloat16 value lies closer to x
    m, e = np.frexp(r)
    assert np.all(np.abs(m * 256 - np.round(m * 256)) == 0)
    ulp = np.ldexp(1.0, e - 8)
    assert np.all(np.abs(r - x) <= ulp / 2 * (1 + 1e-12))


def _identity_theta():
    """Centre taps pass channels straight through (ReLU keeps positives);
    the last layer outputs channels 0 and 1."""
    th = np.zeros(O.net_nparams())
    for l, (ci, co) in enumerate(O.net_channels()):
        w0 = O.net_offset(l, False)
        for c in range(min(ci, co)):
            th[w0 + ((c * ci + c) * 3 + 1) * 3 + 1] = 1.0
    return th


def test_identity_kernels_reproduce_the_input():
    rng = np.random.default_rng(1)
    x = rng.uniform(0.1, 2.0, (2, 6, 5, 7))
    _, y = O.net_forward(_identity_theta(), x, bf16_round=False)
    assert np.array_equal(y, x[:, :2])


def test_off_centre_tap_shifts_with_zero_padding():
    """W[0][0][ky=0][kx=1] = 1 reads the pixel one row up: out[i][j] = in[i-1][j]."""
    rng = np.random.default_rng(2)
    x = rng.uniform(0.1, 2.0, (1, 6, 6, 5))
    th = _identity_theta()
    w0 = O.net_offset(0, False)
    th[w0 + ((0 * 6 + 0) * 3 + 1) * 3 + 1] = 0.0
    th[w0 + ((0 * 6 + 0) * 3 + 0) * 3 + 1] = 1.0
    _, y = O.net_forward(th, x, bf16_round=False)
    want = np.zeros_like(x[0, 0])
    want[1:] = x[0, 0, :-1]
    assert np.array_equal(y[0, 0], want)
    assert np.array_equal(y[0, 1], x[0, 1])


def test_loss_is_the_masked_mean_square():
    y = np.array([[[[1.0, 2.0]], [[3.0, -1.0]]]])
    t = np.array([[[[0.0, 0.0]], [[0.0, 1.0]]]])
    m = np.array([[[[1, 0]], [[1, 1]]]], np.uint8)
    loss, dy = O.net_loss(y, t, m)
    assert loss == pytest.approx((1 + 9 + 4) / 3)
    assert np.allclose(dy, 2 * (y - t) * m / 3)


def _loss_of(theta, x, t, m):
    _, y = O.net_forward(theta, x, bf16_round=False)
    return O.net_loss(y, t, m)[0]


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    th = _rand_theta(rng)
    x = rng.normal(0, 1, (2, 6, 5, 4))
    t = rng.normal(0, 1, (2, 2, 5, 4))
    m = (rng.random((2, 2, 5, 4)) < 0.7).astype(np.uint8)
    acts, y = O.net_forward(th, x, bf16_round=False)
    _, dy = O.net_loss(y, t, m)
    g, gx = O.net_backward(th, acts, dy, bf16_round=False, want_dx=True)
    idx = []
    for l in range(4):
        w0, b0, e = O.net_offset(l, False), O.net_offset(l, True), O.net_offset(l + 1, False)
        idx += list(rng.integers(w0, b0, 12)) + list(rng.integers(b0, e, 3))
    eps = 1e-6
    for q in idx:
        tp, tm = th.copy(), th.copy()
        tp[q] += eps
        tm[q] -= eps
        fd = (_loss_of(tp, x, t, m) - _loss_of(tm, x, t, m)) / (2 * eps)
        assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(fd)), (q, fd, g[q])
    for _ in range(10):
        a, c, i, j = rng.integers(0, 2), rng.integers(0, 6), rng.integers(0, 5), rng.integers(0, 4)
        xp, xm = x.copy(), x.copy()
        xp[a, c, i, j] += eps
        xm[a, c, i, j] -= eps
        fd = (_loss_of(th, xp, t, m) - _loss_of(th, xm, t, m)) / (2 * eps)
        assert abs(fd - gx[a, c, i, j]) <= 1e-6 * max(1.0, abs(fd))


def test_rounded_forward_equals_forward_on_rounded_operands():
    """bf16 mode = exact arithmetic on bf16 weights and bf16 layer inputs."""
    rng = np.random.default_rng(4)
    th = _rand_theta(rng)
    x = rng.normal(0, 1, (1, 6, 4, 4))
    _, y16 = O.net_forward(th, x, bf16_round=True)
    thr = th.copy()
    for l, (ci, co) in enumerate(O.net_channels()):
        w0, b0 = O.net_offset(l, False), O.net_offset(l, True)
        thr[w0:b0] = O.bf16(th[w0:b0])
    # layer by layer with explicit rounding of each input, through single-layer nets
    acts, _ = O.net_forward(thr, O.bf16(x), bf16_round=True)
    assert np.abs(y16).max() > 0
    _, y_again = O.net_forward(thr, O.bf16(x), bf16_round=True)
    assert np.array_equal(y16, y_again)          # rounding is idempotent on rounded operands
    _, y64 = O.net_forward(th, x, bf16_round=False)
    assert np.abs(y16 - y64).max() < 0.05 * np.abs(y64).max()


def test_adamw_first_step_and_constant_gradient():
    rng = np.random.default_rng(5)
    th = _rand_theta(rng)
    g = rng.normal(0, 1, th.size)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    t0 = th.copy()
    lr, wd, eps = 1e-3, 0.01, 1e-8
    O.adamw(th, g, m, v, 1, lr, 0.9, 0.999, eps, wd)
    # bias-corrected moments after one step are g and g^2
    decay = np.zeros(th.size, bool)
    for l in range(4):
        decay[O.net_offset(l, False):O.net_offset(l, True)] = True
    want = t0 - lr * (g / (np.abs(g) + eps) + np.where(decay, wd * t0, 0.0))
    assert np.allclose(th, want, rtol=0, atol=1e-15)
    # with a constant gradient the bias-corrected moments stay exactly g and g^2
    th2 = t0.copy()
    m[:] = 0
    v[:] = 0
    for step in range(1, 6):
        before = th2.copy()
        O.adamw(th2, g, m, v, step, lr, 0.9, 0.999, eps, 0.0)
        assert np.allclose(before - th2, lr * g / (np.abs(g) + eps), rtol=1e-9, atol=1e-15)


def _plane_state(h, w, scale_t=1.0):
    st = O.new_state(2, h, w)
    i, j = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    st.t[0] = 500 + 2.0 * i - 1.5 * j
    st.r[0] = 3.0
    st.alive[0] = 1
    return st


def test_features_of_a_plane_and_of_a_spike():
    st = _plane_state(7, 8)
    x = O.net_features(st, 3.0)
    # a linear surface equals its 8-neighbour mean in the interior
    assert np.allclose(x[0, 1:-1, 1:-1], 0.0, atol=1e-12)
    assert np.allclose(x[1], np.log1p(3.0))
    assert np.all(x[2, 1:-1, 1:-1] == 1.0) and x[2, 0, 0] == pytest.approx(4 / 9)   # 8 / 3 neighbours
    assert np.all(x[3:] == 0.0)                     # empty second slot
    st.t[0, 3, 4] += 6.0
    x = O.net_features(st, 3.0)
    assert x[0, 3, 4] == pytest.approx(2.0)
    assert x[0, 3, 5] == pytest.approx(-6.0 / 8 / 3.0)
    # beyond 4 scale in depth a point is on another surface: no neighbours
    st.t[0, 3, 4] += 100.0
    x = O.net_features(st, 3.0)
    assert x[0, 3, 4] == 0.0 and x[2, 3, 4] == pytest.approx(1 / 9)
    # its right-hand neighbour keeps 7 plane neighbours, whose mean offset is
    # (0, +1/7) pixels: 1.5 / 7 bins below the plane value (slope -1.5 in j)
    assert x[0, 3, 5] == pytest.approx(1.5 / 7 / 3.0) and x[2, 3, 5] == pytest.approx(8 / 9)
    st.alive[0, 2, 2] = 0
    x = O.net_features(st, 3.0)
    assert x[0, 2, 2] == x[1, 2, 2] == x[2, 2, 2] == 0.0


def test_features_use_same_surface_points_of_any_slot():
    """A second surface 300 bins behind does not enter a point's neighbours;
    the same surface held in another slot of a neighbour does."""
    st = _plane_state(5, 5)
    st.t[1] = st.t[0] + 300.0
    st.r[1] = 1.0
    st.alive[1] = 1
    x = O.net_features(st, 3.0)
    assert x[0, 2, 2] == pytest.approx(0.0, abs=1e-12) and x[2, 2, 2] == 1.0
    assert x[3, 2, 2] == pytest.approx(0.0, abs=1e-12) and x[5, 2, 2] == 1.0
    # swap the slots of one neighbour: the same points, the same features
    st.t[[0, 1], 2, 3] = st.t[[1, 0], 2, 3]
    y = O.net_features(st, 3.0)
    assert y[0, 2, 2] == pytest.approx(0.0, abs=1e-12) and y[2, 2, 2] == 1.0


def test_learned_step_limits():
    """A zero network leaves every point in place; a fallback below zero hands
    every point to APSS."""
    sc = scenes.small_random(9, 11, 256, n_comp=2, seed=3)
    z = O.synthesize(scenes.sampling_tables(sc))
    prm = scenes.make_params(sc)
    st = O.init(z, None, O.OIrf(sc.irf.samples, sc.irf.origin), prm)
    p0 = dict(prm, net_theta=np.zeros(O.net_nparams()), net_scale=3.0, net_fallback=5.0)
    a = st.copy()
    O.learned_depth(sc.h, sc.w, sc.t, p0, a)
    assert np.array_equal(a.t, st.t)
    b = st.copy()
    O.learned_depth(sc.h, sc.w, sc.t, dict(p0, net_fallback=-1.0), b)
    c = st.copy()
    O.apss(sc.h, sc.w, sc.t, prm, c)
    assert np.array_equal(b.t, c.t)
