"""GPU (sm_103a) kernels vs the FP64 oracle, through the C ABI.

Integer work (photon synthesis, sparse compaction, matched filter, peak bins)
must be bit-exact; floating-point results within 1e-3 bins of depth and 1e-4
relative intensity/background of the oracle (the FP32 tolerance)."""
import numpy as np
import pytest

import scenes
from gpu_util import (compare_clouds, make_ctx, np_of, oracle_irf, oracle_with_probes,
                      state_f32_rounded, state_to_device, torch_mod, u16_np, upload_u16,
                      workload_params)

pytestmark = pytest.mark.gpu

TOL_T = 1e-3
TOL_R = 1e-4


def _scenes_small():
    return [
        scenes.plane_hemisphere(),                                   # 32x32x1024, K=1
        scenes.small_random(13, 29, 300, n_comp=2, seed=4),          # ragged tile edges
        scenes.small_random(1, 1, 64, n_comp=1, seed=5),             # single pixel
        scenes.small_random(1, 37, 203, n_comp=2, seed=6),           # one row, T % 8 != 0
        scenes.small_random(9, 17, 129, n_comp=3, seed=7),
    ]


@pytest.mark.parametrize("idx", range(5))
def test_synthesis_bit_exact(orc, idx):
    sc = _scenes_small()[idx]
    tab = scenes.sampling_tables(sc)
    ctx = make_ctx(sc)
    z = u16_np(ctx.synthesize(tab))
    assert np.array_equal(z, orc.synthesize(tab))


def test_synthesis_bit_exact_multisurface_full_size(orc):
    sc = scenes.net_object_wall()                                    # 141x141x4096
    tab = scenes.sampling_tables(sc)
    ctx = make_ctx(sc)
    z = u16_np(ctx.synthesize(tab))
    assert np.array_equal(z, orc.synthesize(tab))


@pytest.mark.parametrize("idx", range(5))
def test_compaction_bit_exact(orc, idx):
    sc = _scenes_small()[idx]
    tab = scenes.sampling_tables(sc)
    z = orc.synthesize(tab)
    ctx = make_ctx(sc)
    off, ent = ctx.compact(upload_u16(z))
    off = off.cpu().numpy().view(np.uint32)
    ent = ent.cpu().numpy().view(np.uint32)
    fr = orc.OFrame(z)
    assert np.array_equal(off, fr.off.astype(np.uint32))
    assert np.array_equal(ent >> 16, fr.bin.astype(np.uint32))
    assert np.array_equal(ent & 0xFFFF, fr.cnt.astype(np.uint32))


@pytest.mark.parametrize("idx", range(5))
def test_matched_filter_bit_exact(orc, idx):
    sc = _scenes_small()[idx]
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc)
    ctx = make_ctx(sc)
    y = ctx.lmf(prm, dense=upload_u16(z)).cpu().numpy()
    irf = oracle_irf(orc, sc)
    kern = orc.lmf_kernel(irf, prm["lmf_delta_rel"], prm["lmf_frac_bits"])
    for i in range(sc.h):
        for j in range(sc.w):
            want, _ = orc.lmf(z[i, j], kern, irf.origin)
            assert np.array_equal(y[i, j], want), (i, j)


def _init_pair(orc, sc, **over):
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc, **over)
    ctx = make_ctx(sc, k=prm["k_max"])
    g = np_of(ctx.init(prm, dense=upload_u16(z)))
    o = orc.init(z, None, oracle_irf(orc, sc), prm)
    return z, prm, ctx, g, o


@pytest.mark.parametrize("idx", range(5))
def test_init_peaks_bit_exact(orc, idx):
    sc = _scenes_small()[idx]
    z, prm, ctx, g, o = _init_pair(orc, sc)
    assert np.array_equal(g["alive"], o.alive)
    assert np.array_equal(g["t"].astype(np.float64), o.t)       # integer peak bins
    np.testing.assert_allclose(g["r"], o.r, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(g["b"], o.b, rtol=1e-5, atol=1e-12)
    assert g["n_points"] == int(o.alive.sum())
    # the sparse list built inside the initialisation kernel
    seg, ent, used = ctx.get_sparse(sc.h * sc.w, int(np.count_nonzero(z)))
    assert used == np.count_nonzero(z)
    fr = orc.OFrame(z)
    for p in range(sc.h * sc.w):
        s, n = seg[p]
        e = ent[s:s + n]
        assert np.array_equal(e >> 16, fr.bin[fr.off[p]:fr.off[p + 1]])
        assert np.array_equal(e & 0xFFFF, fr.cnt[fr.off[p]:fr.off[p + 1]])


def test_init_multisurface_full_size_bit_exact(orc):
    sc = scenes.net_object_wall()
    z, prm, ctx, g, o = _init_pair(orc, sc)
    assert np.array_equal(g["alive"], o.alive)
    assert np.array_equal(g["t"].astype(np.float64), o.t)
    np.testing.assert_allclose(g["r"], o.r, rtol=1e-5, atol=1e-6)


def _phase_setup(orc, sc, **over):
    torch = torch_mod()
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc, **over)
    irf = oracle_irf(orc, sc)
    st0 = state_f32_rounded(orc, orc.init(z, None, irf, prm))
    ctx = make_ctx(sc, k=prm["k_max"])
    off, ent = ctx.compact(upload_u16(z))
    return z, prm, irf, st0, ctx, (off, ent), orc.OFrame(z)


@pytest.mark.parametrize("idx", [0, 1, 4])
@pytest.mark.parametrize("bkg_mode", [0, 1])
def test_phase_a_depth_step(orc, idx, bkg_mode):
    sc = _scenes_small()[idx]
    z, prm, irf, st0, ctx, csr, fr = _phase_setup(orc, sc, bkg_mode=bkg_mode)
    for first in (1, 0):
        dev = state_to_device(st0)
        ctx.phase(0, first, prm, csr, dev, shape=(sc.h, sc.w, sc.t))
        g = np_of(dev)
        o = st0.copy()
        if not first:
            orc.bkg_lowpass(sc.h, sc.w, prm, o.b)
        orc.t_step(fr, irf, prm, o)
        compare_clouds(g, o, sc.t, TOL_T, TOL_R, label=f"A first={first}")


@pytest.mark.parametrize("idx", [0, 1, 4])
@pytest.mark.parametrize("den,fp64", [(1, 0), (0, 0), (1, 1), (3, 0), (4, 0)])
def test_phase_b_apss_and_intensity_step(orc, idx, den, fp64):
    """Phase B with each depth denoiser (none, APSS with its solve in FP32 or
    FP64, plane fit, bilateral) then the intensity step, from identical inputs."""
    sc = _scenes_small()[idx]
    z, prm, irf, st0, ctx, csr, fr = _phase_setup(orc, sc, depth_denoiser=den, apss_fp64=fp64)
    # start from a state after one depth step so that APSS has work to do
    orc.t_step(fr, irf, prm, st0)
    st0 = state_f32_rounded(orc, st0)
    dev = state_to_device(st0)
    ctx.phase(1, 0, prm, csr, dev, shape=(sc.h, sc.w, sc.t))
    g = np_of(dev)
    o = st0.copy()
    orc.depth_denoise(sc.h, sc.w, sc.t, prm, o)
    orc.r_step(fr, irf, prm, o)
    compare_clouds(g, o, sc.t, TOL_T, TOL_R, label=f"B den={den} fp64={fp64}")


@pytest.mark.parametrize("idx", [0, 1, 4])
@pytest.mark.parametrize("den", [1, 0])
def test_phase_c_intensity_lowpass_prune_and_background_step(orc, idx, den):
    sc = _scenes_small()[idx]
    z, prm, irf, st0, ctx, csr, fr = _phase_setup(orc, sc, intensity_denoiser=den)
    orc.t_step(fr, irf, prm, st0)
    orc.apss(sc.h, sc.w, sc.t, prm, st0)
    orc.r_step(fr, irf, prm, st0)
    st0 = state_f32_rounded(orc, st0)
    dev = state_to_device(st0)
    ctx.phase(2, 0, prm, csr, dev, shape=(sc.h, sc.w, sc.t))
    g = np_of(dev)
    o = st0.copy()
    orc.int_lowpass(sc.h, sc.w, prm, o)
    orc.b_step(fr, irf, prm, o)
    compare_clouds(g, o, sc.t, TOL_T, TOL_R, label="C")


@pytest.mark.parametrize("idx", range(5))
def test_reconstruct_matches_oracle(orc, idx):
    sc = _scenes_small()[idx]
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc)
    ctx = make_ctx(sc, k=prm["k_max"])
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z)))
    o, probes = oracle_with_probes(orc, sc, z, prm)
    stats = compare_clouds(g, o, sc.t, TOL_T, TOL_R, probes=probes, max_ill_frac=0.05,
                           label=sc.name, r_min=prm["r_min"])
    assert g["n_points"] == int(g["alive"].sum())
    print(sc.name, stats)


@pytest.mark.parametrize("over", [dict(bkg_mode=1), dict(depth_denoiser=0, intensity_denoiser=0),
                                  dict(apss_fp64=1), dict(depth_denoiser=3), dict(depth_denoiser=4),
                                  dict(k_max=4), dict(k_max=1, win_r=1), dict(n_iter=0),
                                  dict(win_r=4, apss_radius=72.0, int_radius=72.0)])
def test_reconstruct_options_match_oracle(orc, over):
    sc = scenes.small_random(21, 19, 256, n_comp=2, seed=11)
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc, **over)
    ctx = make_ctx(sc, k=prm["k_max"])
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z)))
    o, probes = oracle_with_probes(orc, sc, z, prm)
    stats = compare_clouds(g, o, sc.t, TOL_T, TOL_R, probes=probes, max_ill_frac=0.05,
                           label=str(over), r_min=prm["r_min"])
    print(over, stats)


def test_reconstruct_with_gain_and_dead_pixels(orc):
    sc = scenes.small_random(16, 24, 256, n_comp=2, seed=12)
    z = orc.synthesize(scenes.sampling_tables(sc))
    rng = np.random.default_rng(0)
    gain = rng.uniform(0.6, 1.4, (sc.h, sc.w)).astype(np.float32)
    gain[3, 5] = 0.0
    gain[10, 0] = 0.0
    torch = torch_mod()
    prm = workload_params(sc)
    ctx = make_ctx(sc, k=prm["k_max"])
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z), gain=torch.from_numpy(gain).cuda()))
    o, probes = oracle_with_probes(orc, sc, z, prm, gain=gain.astype(np.float64))
    compare_clouds(g, o, sc.t, TOL_T, TOL_R, probes=probes, max_ill_frac=0.05, label="gain",
                   r_min=prm["r_min"])
    assert not g["alive"][:, 3, 5].any() and not g["alive"][:, 10, 0].any()


def test_sparse_input_equals_dense_input(orc):
    sc = scenes.small_random(13, 29, 300, n_comp=2, seed=4)
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc)
    ctx = make_ctx(sc, k=prm["k_max"])
    zd = upload_u16(z)
    a = np_of(ctx.reconstruct(prm, dense=zd))
    csr = ctx.compact(zd)
    b = np_of(ctx.reconstruct(prm, csr=csr, shape=z.shape))
    for k in ("t", "r", "alive", "b"):
        assert np.array_equal(a[k], b[k]), k


def test_batch_results_equal_single_frame_results(orc):
    """Frames of mixed sizes in one batched call give bitwise the results of
    reconstructing each alone."""
    scs = [scenes.small_random(13, 29, 300, n_comp=2, seed=21),
           scenes.small_random(32, 32, 256, n_comp=2, seed=22),
           scenes.small_random(5, 70, 200, n_comp=2, seed=23),
           scenes.small_random(1, 1, 64, n_comp=2, seed=24)]
    irf = scenes.gaussian_irf(3.0, 12)
    for s in scs:
        s.irf = irf
    zs = [orc.synthesize(scenes.sampling_tables(s)) for s in scs]
    prm = workload_params(scs[0])
    from paper_1905_06700_b300 import rt3d as R
    ctx = R.Context(32, 70, 300, 2, irf.samples, irf.origin, max_batch=8)
    singles = [np_of(ctx.reconstruct(prm, dense=upload_u16(z))) for z in zs]
    batch = [np_of(o) for o in ctx.reconstruct_batch(prm, [dict(dense=upload_u16(z)) for z in zs])]
    for s, b in zip(singles, batch):
        for k in ("t", "r", "alive", "b", "n_points"):
            assert np.array_equal(np.asarray(s[k]), np.asarray(b[k])), k


def test_largest_batch_equals_single_frames(orc):
    """The largest batch (64 frames) of ragged sizes in one call (two chains of frames
    in the captured graph) give bitwise the single-frame results."""
    from paper_1905_06700_b300 import rt3d as R
    irf = scenes.gaussian_irf(3.0, 12)
    scs = []
    for i in range(R.MAX_BATCH):
        s = scenes.small_random(3 + i % 7, 5 + (i * 3) % 11, 128, n_comp=2, seed=100 + i)
        s.irf = irf
        scs.append(s)
    zs = [orc.synthesize(scenes.sampling_tables(s)) for s in scs]
    prm = workload_params(scs[0])
    ctx = R.Context(9, 15, 128, 2, irf.samples, irf.origin, max_batch=len(scs))
    frames = [dict(dense=upload_u16(z)) for z in zs]
    batch = [np_of(o) for o in ctx.reconstruct_batch(prm, frames)]
    assert ctx.device_status() == R.RT3D_OK
    for z, b in zip(zs, batch):
        s = np_of(ctx.reconstruct(prm, dense=upload_u16(z)))
        for k in ("t", "r", "alive", "b", "n_points"):
            assert np.array_equal(np.asarray(s[k]), np.asarray(b[k])), k


def test_host_entry_point_equals_device_path(orc):
    from paper_1905_06700_b300 import rt3d as R
    sc = scenes.small_random(13, 29, 300, n_comp=2, seed=4)
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc)
    ctx = make_ctx(sc, k=prm["k_max"])
    a = np_of(ctx.reconstruct(prm, dense=upload_u16(z)))
    b = R.reconstruct_host(ctx, prm, z)
    for k in ("t", "r", "alive", "b"):
        assert np.array_equal(a[k], b[k]), k
    assert int(b["n_points"][0]) == a["n_points"]


def test_batched_host_entry_point_equals_device_path(orc):
    """Ragged frames in host buffers (dense, sparse, and with a gain map) through
    rt3d_reconstruct_batch_host: bit for bit the device-resident batch."""
    from paper_1905_06700_b300 import rt3d as R
    torch = torch_mod()
    scs = [scenes.small_random(13, 29, 300, n_comp=2, seed=4), scenes.small_random(17, 11, 300, n_comp=1, seed=5),
           scenes.small_random(9, 21, 300, n_comp=2, seed=6)]
    zs = [orc.synthesize(scenes.sampling_tables(sc)) for sc in scs]
    prm = workload_params(scs[0])
    ctx = make_ctx(scs[0], k=prm["k_max"], max_h=17, max_w=29, max_batch=3)
    gain = np.random.default_rng(7).uniform(0.5, 1.5, (9, 21)).astype(np.float32)
    dev = ctx.reconstruct_batch(prm, [dict(dense=upload_u16(zs[0])), dict(dense=upload_u16(zs[1])),
                                      dict(dense=upload_u16(zs[2]), gain=torch.from_numpy(gain).cuda())])
    off, ent = ctx.compact(upload_u16(zs[1]))
    csr = (off.cpu().numpy().astype(np.uint32), ent.cpu().numpy().astype(np.uint32), zs[1].shape)
    host = R.reconstruct_batch_host(ctx, prm, [dict(dense=zs[0]), dict(csr=csr), dict(dense=zs[2], gain=gain)])
    for i in range(3):
        a = np_of(dev[i])
        for k in ("t", "r", "alive", "b"):
            assert np.array_equal(a[k], host[i][k]), (i, k)
        assert int(host[i]["n_points"][0]) == a["n_points"]


def test_batched_host_entry_point_in_copy_groups_equals_device_path(orc):
    """Dense frames of 64 MiB and more: rt3d_reconstruct_batch_host copies them
    in groups on its own stream while earlier groups are reconstructed (five
    frames: four groups of 1, 1, 1 and 2); cold start, then a warm start from
    those results, bit for bit the device-resident batch."""
    from paper_1905_06700_b300 import rt3d as R
    torch = torch_mod()
    scs = [scenes.small_random(128, 128, 2048, n_comp=2, seed=60 + i) for i in range(5)]
    for sc in scs[1:]:
        sc.irf = scs[0].irf
    prm = workload_params(scs[0], n_iter=4)
    ctx = make_ctx(scs[0], k=prm["k_max"], max_batch=5)
    dense = [ctx.synthesize(scenes.sampling_tables(sc)) for sc in scs]
    host_z = [u16_np(d) for d in dense]
    assert host_z[0].nbytes >= 64 << 20
    dev = ctx.reconstruct_batch(prm, [dict(dense=d) for d in dense])
    host = R.reconstruct_batch_host(ctx, prm, [dict(dense=z) for z in host_z])
    for i in range(5):
        a = np_of(dev[i])
        for k in ("t", "r", "alive", "b"):
            assert np.array_equal(a[k], host[i][k]), (i, k)
        assert int(host[i]["n_points"][0]) == a["n_points"]
    warm = dict(prm, warm_start=1)
    dev = ctx.reconstruct_batch(warm, [dict(dense=d) for d in dense], outs=dev)
    host = R.reconstruct_batch_host(ctx, warm, [dict(dense=z) for z in host_z], outs=host)
    torch.cuda.synchronize()
    for i in range(5):
        a = np_of(dev[i])
        for k in ("t", "r", "alive", "b"):
            assert np.array_equal(a[k], host[i][k]), (i, k)


def test_capacity_overflow_is_reported_not_faulted(orc):
    from paper_1905_06700_b300 import rt3d as R
    sc = scenes.small_random(16, 16, 256, n_comp=2, seed=3)
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc)
    ctx = make_ctx(sc, k=prm["k_max"], max_entries=int(np.count_nonzero(z)) // 2)
    ctx.reconstruct(prm, dense=upload_u16(z))
    assert ctx.device_status() == R.RT3D_E_CAPACITY
    assert ctx.device_status() == R.RT3D_OK          # cleared after reading
    ctx2 = make_ctx(sc, k=prm["k_max"])
    ctx2.reconstruct(prm, dense=upload_u16(z))
    assert ctx2.device_status() == R.RT3D_OK


def test_dense_pixels_init_and_reconstruct_match_oracle(orc):
    """Pixels with ~400 nonzero bins of 1024 (background 0.5 photons per bin):
    more entries than the init's per-warp stage holds (re-read and emitted to
    global memory), one cluster spanning the whole histogram (several filter
    chunks), the multi-round cluster search, and long bin runs per lane in the
    loop's sums."""
    sc = scenes.small_random(12, 10, 1024, n_comp=2, seed=31, mean_signal=50.0, bkg=0.5)
    z, prm, ctx, g, o = _init_pair(orc, sc)
    nnz = np.count_nonzero(z, axis=2)
    assert nnz.min() > 256
    assert np.array_equal(g["alive"], o.alive)
    assert np.array_equal(g["t"].astype(np.float64), o.t)
    np.testing.assert_allclose(g["r"], o.r, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(g["b"], o.b, rtol=1e-5, atol=1e-12)
    seg, ent, used = ctx.get_sparse(sc.h * sc.w, int(nnz.sum()))
    assert used == int(nnz.sum())
    fr = orc.OFrame(z)
    for p in range(sc.h * sc.w):
        s, n = seg[p]
        e = ent[s:s + n]
        assert np.array_equal(e >> 16, fr.bin[fr.off[p]:fr.off[p + 1]])
        assert np.array_equal(e & 0xFFFF, fr.cnt[fr.off[p]:fr.off[p + 1]])
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z)))
    o, probes = oracle_with_probes(orc, sc, z, prm)
    stats = compare_clouds(g, o, sc.t, TOL_T, TOL_R, probes=probes, max_ill_frac=0.05,
                           label="dense pixels", r_min=prm["r_min"])
    print("dense pixels", stats)


def test_longest_histogram_and_irf_match_oracle(orc):
    """The largest histogram and IRF the library accepts (16384 bins, a
    256-sample gamma IRF): eight filter taps per lane, 16-bit bin indices at
    their top, the loop's interval table at its longest."""
    irf = scenes.gamma_irf(6.0, 12.0, 256)
    sc = scenes.small_random(3, 5, 16384, n_comp=2, seed=41, mean_signal=40.0, bkg=0.002, irf=irf)
    z, prm, ctx, g, o = _init_pair(orc, sc)
    assert np.array_equal(g["alive"], o.alive)
    assert np.array_equal(g["t"].astype(np.float64), o.t)
    np.testing.assert_allclose(g["r"], o.r, rtol=1e-5, atol=1e-6)
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z)))
    o, probes = oracle_with_probes(orc, sc, z, prm)
    # depths near 16384 bins are FP32 numbers 2^-9 apart: the depth tolerance
    # is four of those spacings (1e-3 bins is below the format's resolution)
    tol_t = max(TOL_T, 4.0 * float(np.spacing(np.float32(sc.t))))
    stats = compare_clouds(g, o, sc.t, tol_t, TOL_R, probes=probes, max_ill_frac=0.05,
                           label="T=16384, L=256", r_min=prm["r_min"])
    print("T=16384, L=256", stats)


def test_filter_range_guard_is_reported_and_spares_other_pixels(orc):
    """A pixel whose photons times the largest tap reach 2^31 cannot have an
    exact int32 filter: the call reports RT3D_E_RANGE and that pixel keeps no
    points, while every other pixel equals the oracle's."""
    from paper_1905_06700_b300 import rt3d as R
    sc = scenes.small_random(6, 7, 512, n_comp=2, seed=43)
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc)
    kern = orc.lmf_kernel(oracle_irf(orc, sc), prm["lmf_delta_rel"], prm["lmf_frac_bits"])
    z[2, 3, :] = 65535
    assert int(z[2, 3].sum()) * int(np.abs(kern).max()) >= 2 ** 31
    ctx = make_ctx(sc, k=prm["k_max"])
    g = np_of(ctx.init(prm, dense=upload_u16(z)))
    assert ctx.device_status() == R.RT3D_E_RANGE
    assert not g["alive"][:, 2, 3].any()
    o = orc.init(z, None, oracle_irf(orc, sc), prm)
    keep = np.ones((sc.h, sc.w), bool)
    keep[2, 3] = False
    assert np.array_equal(g["alive"][:, keep], o.alive[:, keep])
    assert np.array_equal(g["t"][:, keep].astype(np.float64), o.t[:, keep])


def test_warm_start_on_a_moving_scene_matches_oracle(orc):
    """A stream's next frame (the scene moved by one bin) started from the
    previous frame's cloud: the GPU's warm start against the oracle's loop run
    from the same state (every value rounded through float32, as the GPU
    holds it), with the same perturbation probe for ill-conditioned points."""
    base = scenes.small_random(14, 23, 300, n_comp=2, seed=71)
    sc1, sc2 = scenes.moving_frame(base, 0), scenes.moving_frame(base, 1)
    z1 = orc.synthesize(scenes.sampling_tables(sc1))
    z2 = orc.synthesize(scenes.sampling_tables(sc2))
    prm = workload_params(base)
    ctx = make_ctx(base, k=prm["k_max"])
    g1 = ctx.reconstruct(prm, dense=upload_u16(z1))
    a = np_of(g1)
    start = orc.new_state(prm["k_max"], base.h, base.w)
    start.t[:] = a["t"]
    start.r[:] = a["r"]
    start.alive[:] = a["alive"]
    start.b[:] = a["b"]
    g2 = np_of(ctx.reconstruct(dict(prm, warm_start=1), dense=upload_u16(z2), out=g1))
    from oracle import compare
    o, probes = compare.palm_with_probes(orc.OFrame(z2), oracle_irf(orc, base), prm, start, prm["n_iter"])
    stats = compare_clouds(g2, o, base.t, TOL_T, TOL_R, probes=probes, max_ill_frac=0.05, label="warm start",
                           r_min=prm["r_min"])
    print("warm start", stats)


def test_empty_histograms_give_no_points(orc):
    sc = scenes.small_random(7, 9, 128, n_comp=1, seed=1)
    z = np.zeros((sc.h, sc.w, sc.t), np.uint16)
    prm = workload_params(sc)
    ctx = make_ctx(sc, k=prm["k_max"])
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z)))
    assert g["n_points"] == 0 and not g["alive"].any()
    np.testing.assert_allclose(g["b"], np.float32(prm["b_floor"]))


def test_reconstruct_multisurface_full_size_matches_oracle(orc):
    """The benchmark workload (141 x 141 x 4096, up to three surfaces per pixel)
    at full size, every point compared."""
    sc = scenes.net_object_wall()
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc)
    ctx = make_ctx(sc, k=prm["k_max"])
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z)))
    o, probes = oracle_with_probes(orc, sc, z, prm)
    stats = compare_clouds(g, o, sc.t, TOL_T, TOL_R, probes=probes, max_ill_frac=0.05,
                           label="full", r_min=prm["r_min"])
    print("141x141x4096", stats)


@pytest.mark.parametrize("fp64", [1, 0])
def test_two_layer_full_size_matches_oracle(orc, fp64):
    """The precision form's workload at full size (256 x 256 x 4096, two
    surfaces per pixel at a signal-to-background ratio of 0.1: ~54 nonzero
    bins per pixel), every point compared with the FP64 oracle.  This form
    solves the APSS normal equations in FP64 (apss_fp64 = 1) and is held to
    the FP32 tolerance.  With the solve in FP32, the normal equations of a
    few near-planar windows are ill-conditioned enough to move a point by
    about 1e-3 bins more: that variant's error is stated (printed) and
    bounded at 1e-2 bins.  The BF16 and FP16 tensor-core filters give the
    integer path's results bit for bit (test_gpu_tc), so they inherit these
    figures."""
    sc = scenes.two_layer()
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc, apss_fp64=fp64)
    ctx = make_ctx(sc, k=prm["k_max"])
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z)))
    o, probes = oracle_with_probes(orc, sc, z, prm)
    stats = compare_clouds(g, o, sc.t, TOL_T if fp64 else 1e-2, TOL_R, probes=probes, max_ill_frac=0.05,
                           label=f"two_layer 256x256x4096 apss_fp64={fp64}", r_min=prm["r_min"])
    print("256x256x4096 SBR 0.1, APSS solve in", "FP64" if fp64 else "FP32", stats)


@pytest.mark.parametrize("den,fp64", [(1, 0), (1, 1), (3, 0), (4, 0)])
def test_phase_b_full_frame_each_denoiser(orc, den, fp64):
    """One phase B (depth denoiser, then the intensity step) on the full
    141 x 141 x 4096 benchmark frame, from the oracle's own state after five
    iterations (rounded to float32), for APSS (solve in FP32 and FP64), the
    plane fit and the bilateral filter: every depth within a few float32
    spacings of the oracle's step, every intensity within 1e-4."""
    sc = scenes.net_object_wall()
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc, depth_denoiser=den, apss_fp64=fp64)
    irf = oracle_irf(orc, sc)
    fr = orc.OFrame(z)
    st = orc.init(z, None, irf, prm)
    orc.palm(fr, irf, prm, st, 5)
    orc.t_step(fr, irf, prm, st)
    st = state_f32_rounded(orc, st)
    ctx = make_ctx(sc, k=prm["k_max"])
    csr = ctx.compact(upload_u16(z))
    dev = state_to_device(st)
    ctx.phase(1, 0, prm, csr, dev, shape=(sc.h, sc.w, sc.t))
    g = np_of(dev)
    o = st.copy()
    orc.depth_denoise(sc.h, sc.w, sc.t, prm, o)
    orc.r_step(fr, irf, prm, o)
    a = o.alive.astype(bool)
    dt = np.abs(g["t"].astype(np.float64) - o.t)[a]
    spacing = np.spacing(np.abs(o.t[a]).astype(np.float32)).astype(np.float64)
    dr = (np.abs(g["r"].astype(np.float64) - o.r) / np.maximum(o.r, 0.1))[a]
    print(f"phase B full frame den={den} fp64={fp64}: max |dt| {dt.max():.3e} bins "
          f"({(dt / spacing).max():.2f} float32 spacings), max rel |dr| {dr.max():.2e}")
    assert np.all(dt <= 4.0 * spacing)
    assert dr.max() <= TOL_R
