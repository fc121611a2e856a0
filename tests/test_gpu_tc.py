"""Tensor-core log-matched filter (lmf_precision BF16 / FP16) vs the FP64
oracle and vs the CUDA-core integer path, through the C ABI.

The filter output is an integer either way (counts and quantised taps are
exact operands, every partial sum an exact multiple of the accumulator unit),
so the matched filter and the peak bins must be bit-exact against the oracle
and the whole reconstruction bitwise equal to the integer path's."""
import numpy as np
import pytest

import scenes
from gpu_util import make_ctx, np_of, oracle_irf, torch_mod, upload_u16, workload_params

pytestmark = pytest.mark.gpu

MODES = {"bf16": 1, "fp16": 2}


def _scenes_tc():
    return [
        scenes.plane_hemisphere(),                                             # 32x32x1024: 8 tiles
        scenes.small_random(13, 29, 256, n_comp=2, seed=4),                    # 377 px: ragged last tile
        scenes.small_random(1, 1, 64, n_comp=1, seed=5),                       # single pixel, one block
        scenes.small_random(9, 17, 200, n_comp=3, seed=7),                     # T not a multiple of 64
        scenes.small_random(5, 30, 512, n_comp=2, seed=8, irf=scenes.gamma_irf(3, 5, 80)),   # 4 offsets
    ]


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("idx", range(5))
def test_tc_matched_filter_bit_exact(orc, idx, mode):
    sc = _scenes_tc()[idx]
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc, lmf_precision=MODES[mode])
    ctx = make_ctx(sc)
    y = ctx.lmf(prm, dense=upload_u16(z)).cpu().numpy()
    irf = oracle_irf(orc, sc)
    kern = orc.lmf_kernel(irf, prm["lmf_delta_rel"], prm["lmf_frac_bits"])
    for i in range(sc.h):
        for j in range(sc.w):
            want, _ = orc.lmf(z[i, j], kern, irf.origin)
            assert np.array_equal(y[i, j], want), (i, j)
    assert ctx.device_status() == 0


def _same(a, b, keys=("t", "r", "alive", "b", "n_points")):
    for k in keys:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("idx", range(5))
def test_tc_init_bit_exact(orc, idx, mode):
    sc = _scenes_tc()[idx]
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc)
    ctx = make_ctx(sc, k=prm["k_max"])
    ref = np_of(ctx.init(prm, dense=upload_u16(z)))
    g = np_of(ctx.init(dict(prm, lmf_precision=MODES[mode]), dense=upload_u16(z)))
    _same(g, ref)
    o = orc.init(z, None, oracle_irf(orc, sc), prm)
    assert np.array_equal(g["alive"], o.alive)
    assert np.array_equal(g["t"].astype(np.float64), o.t)
    assert ctx.device_status() == 0


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("over", [{}, dict(peak_sep=32), dict(peak_sep=1, peak_min_photons=0),
                                  dict(k_max=4, peak_min_photons=3)])
def test_tc_peak_options_bit_exact(orc, mode, over):
    sc = scenes.small_random(11, 23, 320, n_comp=3, seed=31)
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc, **over)
    ctx = make_ctx(sc, k=prm["k_max"])
    ref = np_of(ctx.init(prm, dense=upload_u16(z)))
    g = np_of(ctx.init(dict(prm, lmf_precision=MODES[mode]), dense=upload_u16(z)))
    _same(g, ref)
    o = orc.init(z, None, oracle_irf(orc, sc), prm)
    assert np.array_equal(g["t"].astype(np.float64), o.t)


@pytest.mark.parametrize("mode", sorted(MODES))
def test_tc_reconstruct_equals_integer_path(orc, mode):
    sc = scenes.small_random(21, 19, 256, n_comp=2, seed=11)
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc)
    ctx = make_ctx(sc, k=prm["k_max"])
    zd = upload_u16(z)
    a = np_of(ctx.reconstruct(prm, dense=zd))
    b = np_of(ctx.reconstruct(dict(prm, lmf_precision=MODES[mode]), dense=zd))
    _same(a, b)
    # a warm start (compaction only) in the same mode
    c1 = ctx.reconstruct(dict(prm, lmf_precision=MODES[mode]), dense=zd)
    w1 = np_of(ctx.reconstruct(dict(prm, lmf_precision=MODES[mode], warm_start=1), dense=zd, out=c1))
    c0 = ctx.reconstruct(prm, dense=zd)
    w0 = np_of(ctx.reconstruct(dict(prm, warm_start=1), dense=zd, out=c0))
    _same(w0, w1)


@pytest.mark.parametrize("mode", sorted(MODES))
def test_tc_reconstruct_with_gain_and_dead_pixels_equals_integer_path(orc, mode):
    """A per-pixel gain map with dead pixels (gain 0): the tensor-core init's
    b0 and r0 and the loop that follows equal the integer path's bit for bit."""
    torch = torch_mod()
    sc = scenes.small_random(17, 26, 320, n_comp=2, seed=13)
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc)
    rng = np.random.default_rng(17)
    gain = rng.uniform(0.4, 1.6, (sc.h, sc.w)).astype(np.float32)
    gain[rng.random((sc.h, sc.w)) < 0.05] = 0.0
    ctx = make_ctx(sc, k=prm["k_max"])
    zd = upload_u16(z)
    gd = torch.from_numpy(gain).cuda()
    a = np_of(ctx.reconstruct(prm, dense=zd, gain=gd))
    b = np_of(ctx.reconstruct(dict(prm, lmf_precision=MODES[mode]), dense=zd, gain=gd))
    _same(a, b)
    assert not a["alive"][:, gain == 0].any()


def test_tc_full_size_two_layer_equals_integer_path(orc):
    """The precision-form workload (256 x 256 x 4096, two surfaces, SBR 0.1):
    initialisation and reconstruction bitwise equal to the integer path, and
    the initial peaks equal to the oracle's."""
    sc = scenes.two_layer()
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc)
    ctx = make_ctx(sc, k=prm["k_max"])
    zd = upload_u16(z)
    ref_i = np_of(ctx.init(prm, dense=zd))
    o = orc.init(z, None, oracle_irf(orc, sc), prm)
    assert np.array_equal(ref_i["t"].astype(np.float64), o.t)
    for mode in sorted(MODES):
        g = np_of(ctx.init(dict(prm, lmf_precision=MODES[mode]), dense=zd))
        _same(g, ref_i)
    ref = np_of(ctx.reconstruct(prm, dense=zd))
    for mode in sorted(MODES):
        _same(np_of(ctx.reconstruct(dict(prm, lmf_precision=MODES[mode]), dense=zd)), ref)
    assert ctx.device_status() == 0


def test_tc_mixed_batch_equals_integer_path(orc):
    """A batch mixing tensor-core frames with frames the CUDA-core kernel
    initialises (sparse input, a bin count that breaks TMA's 16-byte rows)."""
    irf = scenes.gaussian_irf(3.0, 12)
    scs = [scenes.small_random(13, 29, 256, n_comp=2, seed=21),
           scenes.small_random(32, 32, 256, n_comp=2, seed=22),
           scenes.small_random(5, 70, 203, n_comp=2, seed=23),
           scenes.small_random(9, 9, 64, n_comp=2, seed=24)]
    for s in scs:
        s.irf = irf
    zs = [orc.synthesize(scenes.sampling_tables(s)) for s in scs]
    prm = workload_params(scs[0])
    from paper_1905_06700_b300 import rt3d as R
    ctx = R.Context(32, 70, 256, 2, irf.samples, irf.origin, max_batch=8)
    frames = [dict(dense=upload_u16(z)) for z in zs]
    frames[1] = dict(csr=ctx.compact(upload_u16(zs[1])), shape=zs[1].shape)
    ref = [np_of(o) for o in ctx.reconstruct_batch(prm, frames)]
    for mode in sorted(MODES):
        got = [np_of(o) for o in ctx.reconstruct_batch(dict(prm, lmf_precision=MODES[mode]), frames)]
        for a, b in zip(ref, got):
            _same(a, b)
    assert ctx.device_status() == 0


@pytest.mark.parametrize("mode,limit", [("fp16", 1024), ("bf16", 128)])
def test_tc_count_limit_is_reported(orc, mode, limit):
    """Counts the raw-operand encoding cannot represent raise the range status
    (no fault, no silent error); counts just below the limit stay exact."""
    from paper_1905_06700_b300 import rt3d as R
    sc = scenes.small_random(4, 8, 128, n_comp=1, seed=2)
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc, lmf_precision=MODES[mode])
    ctx = make_ctx(sc, k=prm["k_max"])
    ok = z.copy()
    ok[1, 2, 40] = limit - 1
    y = ctx.lmf(prm, dense=upload_u16(ok)).cpu().numpy()
    irf = oracle_irf(orc, sc)
    kern = orc.lmf_kernel(irf, prm["lmf_delta_rel"], prm["lmf_frac_bits"])
    want, _ = orc.lmf(ok[1, 2], kern, irf.origin)
    assert np.array_equal(y[1, 2], want)
    ctx.init(prm, dense=upload_u16(ok))
    assert ctx.device_status() == R.RT3D_OK
    bad = z.copy()
    bad[1, 2, 40] = limit
    ctx.init(prm, dense=upload_u16(bad))
    assert ctx.device_status() == R.RT3D_E_RANGE


def test_tc_empty_histograms_give_no_points(orc):
    sc = scenes.small_random(7, 9, 128, n_comp=1, seed=1)
    z = np.zeros((sc.h, sc.w, sc.t), np.uint16)
    prm = workload_params(sc, lmf_precision=2)
    ctx = make_ctx(sc, k=prm["k_max"])
    g = np_of(ctx.reconstruct(prm, dense=upload_u16(z)))
    assert g["n_points"] == 0 and not g["alive"].any()
    np.testing.assert_allclose(g["b"], np.float32(prm["b_floor"]))


def test_tc_kernel_is_the_one_that_runs(orc):
    """In a tensor-core mode the dense frames' initialisation is timed under
    the tensor-core kernel and the CUDA-core init does not run."""
    sc = scenes.small_random(16, 16, 256, n_comp=2, seed=3)
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc, lmf_precision=2)
    ctx = make_ctx(sc, k=prm["k_max"])
    ctx.set_profiling(True)
    ctx.kernel_times(reset=True)
    ctx.reconstruct(prm, dense=upload_u16(z))
    kt = ctx.kernel_times(reset=True)
    assert kt["init_tc"][1] == 1 and kt["init"][1] == 0
