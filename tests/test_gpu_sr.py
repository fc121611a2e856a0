"""Super-resolution on the GPU (rt3d_params.upsample) against the FP64 oracle,
through the C ABI: the point-to-cube mapping f sends a u x u window of world
pixels to one lidar pixel (Results, "Observation model"; the 32 x 32 ->
96 x 96 dynamic-scene experiment)."""
import numpy as np
import pytest

import scenes
from gpu_util import compare_clouds, make_ctx, np_of, oracle_irf, torch_mod, upload_u16

pytestmark = pytest.mark.gpu

TOL_T = 1e-3
TOL_R = 1e-4


def sr_params(sc, **over):
    """Parameters of the super-resolved form: denoisers on the world grid
    (pitch 4 bins per world pixel, radius 3.5 world pixels), two points per
    world pixel, u = 3."""
    p = scenes.make_params(sc, pixel_pitch=4.0, k_max=2, upsample=3)
    p.update(over)
    return p


def _frame(orc, h=12, w=10, seed=3):
    sc, _ = scenes.camouflage_people(h, w, 153, up=3, seed=seed)
    return sc, orc.synthesize(scenes.sampling_tables(sc))


def test_sr_init_spreads_peaks_bit_exact(orc):
    sc, z = _frame(orc)
    prm = sr_params(sc)
    ctx = make_ctx(sc, k=2, max_h=3 * sc.h, max_w=3 * sc.w)
    g = np_of(ctx.init(prm, dense=upload_u16(z)))
    o = orc.init(z, None, oracle_irf(orc, sc), prm)
    assert g["t"].shape == (2, 3 * sc.h, 3 * sc.w) and g["b"].shape == (sc.h, sc.w)
    assert np.array_equal(g["alive"], o.alive)
    assert np.array_equal(g["t"].astype(np.float64), o.t)
    np.testing.assert_allclose(g["r"], o.r, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(g["b"], o.b, rtol=1e-5, atol=1e-12)


@pytest.mark.parametrize("over", [dict(), dict(bkg_mode=1), dict(depth_denoiser=0), dict(depth_denoiser=3),
                                  dict(n_iter=1), dict(apss_fp64=1)])
def test_sr_reconstruct_matches_oracle(orc, over):
    from oracle import compare
    sc, z = _frame(orc)
    prm = sr_params(sc, **over)
    ctx = make_ctx(sc, k=2, max_h=3 * sc.h, max_w=3 * sc.w)
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z)))
    o, probes = compare.reconstruct_with_probes(z, oracle_irf(orc, sc), prm)
    st = compare_clouds(g, o, sc.t, TOL_T, TOL_R, probes=probes, max_ill_frac=0.05,
                        label=f"super-resolution {over}", r_min=prm["r_min"])
    assert g["n_points"] == int(g["alive"].sum())
    print("super-resolution", over, st)


def test_sr_full_size_camouflage_matches_oracle(orc):
    """The dynamic-scene shape at full size: 32 x 32 pixels x 153 bins
    (~900 photons per pixel, half of them background) reconstructed on the
    96 x 96 world grid, every point compared."""
    from oracle import compare
    sc, z = _frame(orc, 32, 32, seed=1)
    prm = sr_params(sc)
    ctx = make_ctx(sc, k=2, max_h=96, max_w=96)
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z)))
    o, probes = compare.reconstruct_with_probes(z, oracle_irf(orc, sc), prm)
    st = compare_clouds(g, o, sc.t, TOL_T, TOL_R, probes=probes, max_ill_frac=0.05,
                        label="camouflage 32x32x153 -> 96x96", r_min=prm["r_min"])
    print("camouflage 32x32x153 -> 96x96", st)


def test_sr_batch_equals_single_frames_and_unsupported_paths_say_so(orc):
    torch = torch_mod()
    from paper_1905_06700_b300 import rt3d as R
    scs = [_frame(orc, 12, 10, seed=s) for s in (4, 5)] + [_frame(orc, 7, 9, seed=6)]
    prm = sr_params(scs[0][0])
    ctx = make_ctx(scs[0][0], k=2, max_h=36, max_w=30, max_batch=3)
    frames = [dict(dense=upload_u16(z)) for _, z in scs]
    batch = [np_of(o) for o in ctx.reconstruct_batch(prm, frames)]
    for f, b in zip(frames, batch):
        a = np_of(ctx.reconstruct(prm, **f))
        for k in ("t", "r", "alive", "b", "n_points"):
            assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    with pytest.raises(R.Rt3dError) as e:
        R.reconstruct_host(ctx, prm, scs[0][1])
    assert e.value.status == R.RT3D_E_UNIMPL
    with pytest.raises(R.Rt3dError) as e:            # 4848 world pixels at u = 4 > 3 x 36 x 30
        ctx.reconstruct_batch(dict(prm, upsample=4), frames)
    assert e.value.status == R.RT3D_E_INVALID
    assert ctx.device_status() == R.RT3D_OK


def test_sr_with_gain_map_matches_oracle(orc):
    """Super-resolution with a detector gain map (a dead lidar pixel: its
    block of world pixels keeps no points) against the FP64 oracle."""
    torch = torch_mod()
    from oracle import compare
    sc, z = _frame(orc, 12, 10, seed=8)
    prm = sr_params(sc)
    rng = np.random.default_rng(8)
    gain = rng.uniform(0.7, 1.3, (sc.h, sc.w)).astype(np.float32)
    gain[4, 6] = 0.0
    ctx = make_ctx(sc, k=2, max_h=3 * sc.h, max_w=3 * sc.w)
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z), gain=torch.from_numpy(gain).cuda()))
    o, probes = compare.reconstruct_with_probes(z, oracle_irf(orc, sc), prm, gain=gain.astype(np.float64))
    st = compare_clouds(g, o, sc.t, TOL_T, TOL_R, probes=probes, max_ill_frac=0.05,
                        label="super-resolution, gain map", r_min=prm["r_min"])
    assert not g["alive"][:, 12:15, 18:21].any()
    print("super-resolution, gain map", st)
