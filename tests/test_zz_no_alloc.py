"""The allocation-free entry point (rt3d_reconstruct_noalloc) against the
context-based one.

Some callers cannot allocate device memory while they run; for them the
library keeps the method's scratch in one static device array.  This file is
collected last so that a run stopping at its first failure has already run
every other test; it passes alone in a fresh process as well."""
import numpy as np
import pytest

import scenes
from gpu_util import make_ctx, np_of, torch_mod, upload_u16

pytestmark = pytest.mark.gpu

TOL_T = 1e-3
TOL_R = 1e-4


def _frame_and_params(orc, sc):
    z = orc.synthesize(scenes.sampling_tables(sc))
    return z, scenes.make_params(sc)


def _call_noalloc(sc, dense, prm, R):
    torch = torch_mod()
    k = prm["k_max"]
    out = dict(t=torch.full((k, sc.h, sc.w), -1.0, device="cuda"),
               r=torch.full((k, sc.h, sc.w), -1.0, device="cuda"),
               alive=torch.full((k, sc.h, sc.w), 7, dtype=torch.uint8, device="cuda"),
               b=torch.full((sc.h, sc.w), -1.0, device="cuda"),
               n_points=torch.full((1,), -1, dtype=torch.int32, device="cuda"))
    fr = R.Frame(sc.h, sc.w, sc.t, R._ptr(dense), None, None, None)
    st = R.rt3d_reconstruct_noalloc(sc.irf.samples, sc.irf.origin, fr, prm,
                                    R.Context.result_struct(out))
    assert st == R.RT3D_OK, R.status_str(st)
    torch.cuda.synchronize()
    return np_of(out)


def _close(a, b):
    assert np.array_equal(a["alive"], b["alive"])
    m = a["alive"].astype(bool)
    assert np.abs(a["t"] - b["t"])[m].max(initial=0.0) <= TOL_T
    assert (np.abs(a["r"] - b["r"]) / np.maximum(np.abs(b["r"]), 0.1))[m].max(initial=0.0) <= TOL_R
    assert (np.abs(a["b"] - b["b"]) / np.maximum(np.abs(b["b"]), 1e-12)).max() <= TOL_R
    assert a["n_points"] == b["n_points"]


def test_noalloc_matches_context_entry_point_on_two_calls_in_a_row(orc):
    from paper_1905_06700_b300 import rt3d as R
    cases = [scenes.plane_hemisphere(),                             # 32 x 32 x 1024 = 2^20 bins
             scenes.small_random(21, 37, 512, n_comp=2, seed=9)]    # second call: other size
    for sc in cases:
        z, prm = _frame_and_params(orc, sc)
        dense = upload_u16(z)
        want = np_of(make_ctx(sc, k=prm["k_max"]).reconstruct(prm, dense=dense))
        got = _call_noalloc(sc, dense, prm, R)
        _close(got, want)


def test_noalloc_rejects_frames_beyond_its_static_scratch():
    from paper_1905_06700_b300 import rt3d as R
    torch = torch_mod()
    prm = R.rt3d_default_params()
    big = torch.zeros((64, 64, 1024), dtype=torch.int16, device="cuda")   # 2^22 bins > 2^21
    out = dict(t=torch.zeros((2, 64, 64), device="cuda"), r=torch.zeros((2, 64, 64), device="cuda"),
               alive=torch.zeros((2, 64, 64), dtype=torch.uint8, device="cuda"),
               b=torch.zeros((64, 64), device="cuda"))
    fr = R.Frame(64, 64, 1024, R._ptr(big), None, None, None)
    st = R.rt3d_reconstruct_noalloc(np.ones(9), 4, fr, prm, R.Context.result_struct(out))
    assert st == R.RT3D_E_INVALID
    wide = R.Frame(200, 100, 8, R._ptr(big), None, None, None)              # 20000 px > 16384
    assert R.rt3d_reconstruct_noalloc(np.ones(9), 4, wide, prm,
                                      R.Context.result_struct(out)) == R.RT3D_E_INVALID


def test_noalloc_sparse_input_warm_start_and_gain_match_context(orc):
    """The other branches of the allocation-free call: the caller's own
    sparse list (no entry area of the static array), a warm start from the
    previous result (the caller's buffers read back), and a gain map; each
    against the context entry point."""
    from paper_1905_06700_b300 import rt3d as R
    torch = torch_mod()
    sc = scenes.small_random(19, 23, 300, n_comp=2, seed=61)
    z, prm = _frame_and_params(orc, sc)
    ctx = make_ctx(sc, k=prm["k_max"])
    dense = upload_u16(z)
    off, ent = ctx.compact(dense)
    gain = torch.from_numpy(np.random.default_rng(2).uniform(0.6, 1.4, (sc.h, sc.w)).astype(np.float32)).cuda()
    k = prm["k_max"]

    def run(fr, p, out):
        st = R.rt3d_reconstruct_noalloc(sc.irf.samples, sc.irf.origin, fr, p, R.Context.result_struct(out))
        assert st == R.RT3D_OK, R.status_str(st)
        torch.cuda.synchronize()
        return np_of(out)

    # sparse list
    out = ctx.new_result(sc.h, sc.w, k)
    got = run(R.Frame(sc.h, sc.w, sc.t, None, R._ptr(off), R._ptr(ent), None), prm, out)
    _close(got, np_of(ctx.reconstruct(prm, csr=(off, ent), shape=z.shape)))
    # warm start from that result, dense input with a gain map
    warm = dict(prm, warm_start=1)
    want_dev = ctx.new_result(sc.h, sc.w, k)
    for key in out:
        want_dev[key].copy_(out[key])
    want = np_of(ctx.reconstruct(warm, dense=dense, gain=gain, out=want_dev))
    got = run(R.Frame(sc.h, sc.w, sc.t, R._ptr(dense), None, None, R._ptr(gain)), warm, out)
    _close(got, want)
    assert R.rt3d_noalloc_status() == R.RT3D_OK


def test_noalloc_status_reports_the_exact_range_guard(orc):
    """A pixel whose photons times the largest filter tap reach 2^31 cannot
    be filtered exactly: the allocation-free call keeps no point there and
    its status query reports RT3D_E_RANGE (then reads clean)."""
    from paper_1905_06700_b300 import rt3d as R
    sc = scenes.small_random(6, 7, 512, n_comp=2, seed=43)
    z, prm = _frame_and_params(orc, sc)
    z[2, 3, :] = 65535
    got = _call_noalloc(sc, upload_u16(z), prm, R)
    assert R.rt3d_noalloc_status() == R.RT3D_E_RANGE
    assert R.rt3d_noalloc_status() == R.RT3D_OK
    assert not got["alive"][:, 2, 3].any()
