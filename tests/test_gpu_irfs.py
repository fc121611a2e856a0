"""Per-pixel instrument responses h_{i,j} (Results, "Observation model") on the
GPU against the FP64 oracle, through the C ABI: a context holds several
responses (rt3d_set_irfs) and a frame names each pixel's (irf_index)."""
import dataclasses

import numpy as np
import pytest

import scenes
from gpu_util import compare_clouds, make_ctx, np_of, torch_mod, upload_u16, workload_params

pytestmark = pytest.mark.gpu

TOL_T = 1e-3
TOL_R = 1e-4


def _two_response_frame(orc, seed, h=19, w=23, t=300):
    """A scene observed through two responses: each pixel's histogram drawn
    with its own response (two syntheses of the same scene, picked per pixel
    in 4 x 4-pixel blocks, so the denoisers' windows see both)."""
    base = scenes.small_random(h, w, t, n_comp=2, seed=seed)
    ia, ib = scenes.gaussian_irf(3.0, 12), scenes.gamma_irf(3.0, 2.0, 30)
    za = orc.synthesize(scenes.sampling_tables(dataclasses.replace(base, irf=ia)))
    zb = orc.synthesize(scenes.sampling_tables(dataclasses.replace(base, irf=ib)))
    rng = np.random.default_rng(seed)
    blocks = rng.integers(0, 2, size=((h + 3) // 4, (w + 3) // 4))
    idx = np.kron(blocks, np.ones((4, 4), np.int64))[:h, :w].astype(np.uint8)
    z = np.where(idx[..., None] == 1, zb, za)
    base = dataclasses.replace(base, irf=ia)
    return base, (ia, ib), idx, z


def _ctx(base, irfs, prm, **kw):
    ctx = make_ctx(base, k=prm["k_max"], **kw)
    ctx.set_irfs([(i.samples, i.origin) for i in irfs])
    return ctx


def _oirfs(orc, irfs):
    return [orc.OIrf(i.samples, i.origin) for i in irfs]


def test_per_pixel_responses_init_bit_exact(orc):
    torch = torch_mod()
    base, irfs, idx, z = _two_response_frame(orc, 91)
    prm = workload_params(base)
    ctx = _ctx(base, irfs, prm)
    g = np_of(ctx.init(prm, dense=upload_u16(z), irf_index=torch.from_numpy(idx).cuda()))
    o = orc.init(z, None, _oirfs(orc, irfs), prm, irf_idx=idx)
    assert np.array_equal(g["alive"], o.alive)
    assert np.array_equal(g["t"].astype(np.float64), o.t)       # integer peak bins
    np.testing.assert_allclose(g["r"], o.r, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(g["b"], o.b, rtol=1e-5, atol=1e-12)


@pytest.mark.parametrize("over", [dict(), dict(bkg_mode=1), dict(depth_denoiser=0, intensity_denoiser=0)])
def test_per_pixel_responses_match_oracle(orc, over):
    torch = torch_mod()
    from oracle import compare
    base, irfs, idx, z = _two_response_frame(orc, 92)
    prm = workload_params(base, **over)
    ctx = _ctx(base, irfs, prm)
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z), irf_index=torch.from_numpy(idx).cuda()))
    o, probes = compare.reconstruct_with_probes(z, _oirfs(orc, irfs), prm, irf_idx=idx)
    st = compare_clouds(g, o, base.t, TOL_T, TOL_R, probes=probes, max_ill_frac=0.05,
                        label=f"two responses {over}", r_min=prm["r_min"])
    print("two responses", over, st)


def test_per_pixel_responses_in_batches_and_host_entry(orc):
    """A batch mixing a two-response frame, a frame without an index and a
    frame whose index names response 1 everywhere gives each frame's single
    results bit for bit; the host-buffer entry point gives the device
    path's; a frame with an index in a tensor-core precision mode (which
    takes the CUDA-core filter) gives the integer path's."""
    torch = torch_mod()
    from paper_1905_06700_b300 import rt3d as R
    base, irfs, idx, z = _two_response_frame(orc, 93)
    prm = workload_params(base)
    ctx = _ctx(base, irfs, prm, max_batch=3)
    other = orc.synthesize(scenes.sampling_tables(scenes.small_random(11, 17, 300, n_comp=2, seed=94,
                                                                      irf=irfs[0])))
    ones = np.ones((11, 17), np.uint8)
    frames = [dict(dense=upload_u16(z), irf_index=torch.from_numpy(idx).cuda()),
              dict(dense=upload_u16(other)),
              dict(dense=upload_u16(other), irf_index=torch.from_numpy(ones).cuda())]
    batch = [np_of(o) for o in ctx.reconstruct_batch(prm, frames)]
    singles = [np_of(ctx.reconstruct(prm, **f)) for f in frames]
    for a, b in zip(batch, singles):
        for k in ("t", "r", "alive", "b", "n_points"):
            assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    assert not np.array_equal(singles[1]["t"], singles[2]["t"])      # response 1 differs
    host = R.reconstruct_host(ctx, prm, z, irf_index=idx)
    for k in ("t", "r", "alive", "b"):
        assert np.array_equal(singles[0][k], host[k]), k
    tc = np_of(ctx.reconstruct(dict(prm, lmf_precision=2), **frames[0]))
    for k in ("t", "r", "alive", "b"):
        assert np.array_equal(singles[0][k], tc[k]), k
    assert ctx.device_status() == R.RT3D_OK


def test_set_irfs_validates():
    from paper_1905_06700_b300 import rt3d as R
    base = scenes.small_random(4, 4, 64, n_comp=1, seed=1)
    ctx = make_ctx(base)
    g = scenes.gaussian_irf(3.0, 12)
    for bad in ([], [(g.samples, g.origin)] * 5, [(np.zeros(5), 2)], [(g.samples, 99)],
                [(np.ones(200), 0), (np.ones(60), 0)]):
        with pytest.raises(R.Rt3dError):
            ctx.set_irfs(bad)
    ctx.set_irfs([(np.ones(59), 0)] * 4)          # 4 x (59 + 6) = 260 <= 262


def test_index_past_the_last_response_reads_as_the_last(orc):
    """rt3d_frame.irf_index: an index past the context's last response reads
    as the last one (the header's contract), bit for bit."""
    torch = torch_mod()
    base, irfs, idx, z = _two_response_frame(orc, 95)
    prm = workload_params(base)
    ctx = _ctx(base, irfs, prm)
    zd = upload_u16(z)
    ones = torch.from_numpy(np.ones_like(idx)).cuda()
    ref = np_of(ctx.reconstruct(prm, dense=zd, irf_index=ones))
    for big in (7, 255):
        got = np_of(ctx.reconstruct(prm, dense=zd, irf_index=torch.from_numpy(np.full_like(idx, big)).cuda()))
        for k in ("t", "r", "alive", "b", "n_points"):
            assert np.array_equal(np.asarray(ref[k]), np.asarray(got[k])), (big, k)


def test_per_pixel_responses_with_gain_and_sparse_input_match_oracle(orc):
    """Per-pixel responses together with a gain map holding dead pixels, first
    from the dense histograms against the FP64 oracle, then from the same
    photons as a sparse list (bit for bit the dense path's)."""
    torch = torch_mod()
    from oracle import compare
    base, irfs, idx, z = _two_response_frame(orc, 96)
    prm = workload_params(base)
    rng = np.random.default_rng(96)
    gain = rng.uniform(0.6, 1.4, (base.h, base.w)).astype(np.float32)
    gain[2, 3] = 0.0
    gain[11, 20] = 0.0
    ctx = _ctx(base, irfs, prm)
    zd = upload_u16(z)
    gd = torch.from_numpy(gain).cuda()
    ix = torch.from_numpy(idx).cuda()
    g = np_of(ctx.reconstruct(prm, dense=zd, gain=gd, irf_index=ix))
    o, probes = compare.reconstruct_with_probes(z, _oirfs(orc, irfs), prm, gain=gain.astype(np.float64),
                                                irf_idx=idx)
    st = compare_clouds(g, o, base.t, TOL_T, TOL_R, probes=probes, max_ill_frac=0.05,
                        label="two responses, gain map", r_min=prm["r_min"])
    assert not g["alive"][:, 2, 3].any() and not g["alive"][:, 11, 20].any()
    csr = ctx.compact(zd)
    s = np_of(ctx.reconstruct(prm, csr=csr, shape=z.shape, gain=gd, irf_index=ix))
    for k in ("t", "r", "alive", "b", "n_points"):
        assert np.array_equal(np.asarray(g[k]), np.asarray(s[k])), k
    print("two responses, gain map", st)


def test_warm_start_with_per_pixel_responses_matches_oracle(orc):
    """A stream's next frame (the scene moved by one bin) observed through two
    responses and started from the previous frame's cloud: the GPU's warm
    start against the oracle's loop run from the same (float32) state."""
    torch = torch_mod()
    from oracle import compare
    base = scenes.small_random(15, 21, 300, n_comp=2, seed=97)
    ia, ib = scenes.gaussian_irf(3.0, 12), scenes.gamma_irf(3.0, 2.0, 30)
    rng = np.random.default_rng(97)
    blocks = rng.integers(0, 2, size=((base.h + 3) // 4, (base.w + 3) // 4))
    idx = np.kron(blocks, np.ones((4, 4), np.int64))[:base.h, :base.w].astype(np.uint8)

    def frame(k):
        sk = scenes.moving_frame(base, k)
        za = orc.synthesize(scenes.sampling_tables(dataclasses.replace(sk, irf=ia)))
        zb = orc.synthesize(scenes.sampling_tables(dataclasses.replace(sk, irf=ib)))
        return np.where(idx[..., None] == 1, zb, za)

    z1, z2 = frame(0), frame(1)
    irfs = (ia, ib)
    b0 = dataclasses.replace(base, irf=ia)
    prm = workload_params(b0)
    ctx = _ctx(b0, irfs, prm)
    ix = torch.from_numpy(idx).cuda()
    g1 = ctx.reconstruct(prm, dense=upload_u16(z1), irf_index=ix)
    a = np_of(g1)
    start = orc.new_state(prm["k_max"], base.h, base.w)
    start.t[:] = a["t"]
    start.r[:] = a["r"]
    start.alive[:] = a["alive"]
    start.b[:] = a["b"]
    g2 = np_of(ctx.reconstruct(dict(prm, warm_start=1), dense=upload_u16(z2), out=g1, irf_index=ix))
    o, probes = compare.palm_with_probes(orc.OFrame(z2, None, irf_idx=idx), _oirfs(orc, irfs), prm, start,
                                         prm["n_iter"])
    st = compare_clouds(g2, o, base.t, TOL_T, TOL_R, probes=probes, max_ill_frac=0.05,
                        label="two responses, warm start", r_min=prm["r_min"])
    print("two responses, warm start", st)


def test_learned_form_with_per_pixel_responses_matches_oracle(orc):
    """The learned depth denoiser in a frame with two responses, against the
    FP64 oracle running the same network (its bfloat16 inputs: the bounds of
    the learned form's own parity test)."""
    torch = torch_mod()
    from paper_1905_06700_b300 import learned
    from paper_1905_06700_b300 import rt3d as R
    base, irfs, idx, z = _two_response_frame(orc, 98)
    prm = dict(workload_params(base), depth_denoiser=2)
    th = learned.init_params(9).astype(np.float64)
    th += np.random.default_rng(16).normal(0, 0.02, th.size)
    th = th.astype(np.float32)
    ctx = _ctx(base, irfs, prm)
    net = R.Net(1, base.h, base.w)
    net.set_params(th)
    ctx.set_depth_net(net)
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z), irf_index=torch.from_numpy(idx).cuda()))
    o = orc.reconstruct(z, _oirfs(orc, irfs), dict(prm, net_theta=th.astype(np.float64)), irf_idx=idx)
    both = g["alive"].astype(bool) & o.alive.astype(bool)
    flips = int((g["alive"].astype(bool) != o.alive.astype(bool)).sum())
    dt = np.abs(g["t"].astype(np.float64) - o.t)[both]
    print("learned form, two responses: points", int(o.alive.sum()), "flips", flips,
          "dt median %.2e p99 %.2e max %.2e" % (np.median(dt), np.percentile(dt, 99), dt.max()))
    assert flips <= 0.01 * max(1, int(o.alive.sum()))
    assert np.median(dt) <= 2e-2 and np.percentile(dt, 99) <= 0.2
