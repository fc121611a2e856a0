"""Bounded device-side waits driven to their limit (no GPU fault involved).

The tensor-core kernels (the BF16/FP16 matched filter of the initialisation
and the learned denoiser's pipelined convolution) wait on shared-memory
barriers for their copies and matrix operations.  Every such wait is bounded
by the context's wait limit (rt3d_set_wait_limit, one second by default).
With the limit set to zero a kernel gives up at its first wait that has not
already completed; it must then await its copies and matrix operations in
flight, free its tensor memory, raise RT3D_E_TIMEOUT, and leave the context
usable: the next call with the default limit returns RT3D_OK and results
bitwise equal to a clean run's."""
import numpy as np
import pytest

import scenes
from gpu_util import make_ctx, np_of, upload_u16, workload_params

pytestmark = pytest.mark.gpu


def _same(a, b):
    for k in ("t", "r", "alive", "b", "n_points"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


def test_tc_init_gives_up_at_its_wait_limit_and_the_context_recovers(orc):
    from paper_1905_06700_b300 import rt3d as R
    sc = scenes.small_random(40, 37, 512, n_comp=2, seed=81)          # 12 tiles of 128 pixels
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = workload_params(sc, lmf_precision=2)                        # FP16 tensor-core filter
    ctx = make_ctx(sc, k=prm["k_max"])
    zd = upload_u16(z)
    clean = np_of(ctx.reconstruct(prm, dense=zd))
    assert ctx.device_status() == R.RT3D_OK
    ctx.set_wait_limit(0)
    ctx.reconstruct(prm, dense=zd)
    assert ctx.device_status() == R.RT3D_E_TIMEOUT
    ctx.set_wait_limit(10 ** 9)
    again = np_of(ctx.reconstruct(prm, dense=zd))
    assert ctx.device_status() == R.RT3D_OK
    _same(clean, again)


def test_learned_convolution_gives_up_at_its_wait_limit_and_the_context_recovers(orc):
    from paper_1905_06700_b300 import learned
    from paper_1905_06700_b300 import rt3d as R
    sc = scenes.small_random(21, 19, 256, n_comp=2, seed=82)
    z = orc.synthesize(scenes.sampling_tables(sc))
    prm = dict(workload_params(sc), depth_denoiser=2, n_iter=3)       # integer filter, learned loop
    ctx = make_ctx(sc, k=prm["k_max"])
    net = R.Net(1, sc.h, sc.w)
    net.set_params(learned.init_params(5))
    ctx.set_depth_net(net)
    zd = upload_u16(z)
    clean = np_of(ctx.reconstruct(prm, dense=zd))
    assert ctx.device_status() == R.RT3D_OK
    ctx.set_wait_limit(0)
    ctx.reconstruct(prm, dense=zd)
    assert ctx.device_status() == R.RT3D_E_TIMEOUT
    ctx.set_wait_limit(10 ** 9)
    again = np_of(ctx.reconstruct(prm, dense=zd))
    assert ctx.device_status() == R.RT3D_OK
    _same(clean, again)


def test_wait_limit_is_validated():
    from paper_1905_06700_b300 import rt3d as R
    sc = scenes.small_random(4, 4, 64, n_comp=1, seed=1)
    ctx = make_ctx(sc)
    with pytest.raises(R.Rt3dError):
        ctx.set_wait_limit(-1)
