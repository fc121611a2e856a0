"""Continuous batching on the GPU: frames of several streams of mixed sizes,
served in overlapping batches with warm starts, give each frame exactly the
result it gets reconstructed alone from the same warm-start state."""
import numpy as np
import pytest

import scenes
from gpu_util import np_of, torch_mod

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("learned", [False, True])
def test_served_results_equal_frames_reconstructed_alone(learned):
    torch = torch_mod()
    from paper_1905_06700_b300 import rt3d as R
    from paper_1905_06700_b300.serve import GpuBackend, Request, Server, SlotLimits
    irf = scenes.gaussian_irf(3.0, 12)
    sizes = [(32, 32, 1024), (48, 40, 512), (64, 64, 1024), (20, 70, 256)]
    bases = []
    for s, (h, w, t) in enumerate(sizes):
        sc = scenes.small_random(h, w, t, n_comp=2, seed=40 + s)
        sc.irf = irf
        bases.append(sc)
    prm = scenes.make_params(bases[0], n_iter=8)
    net = None
    if learned:
        # the learned form: a network (random weights suffice for the invariance)
        from paper_1905_06700_b300 import learned as L
        net = R.Net(1, 64, 70)
        net.set_params(L.init_params(1))
        prm = dict(prm, depth_denoiser=2)
    lim = SlotLimits(max_frames=3, max_pixels=3 * 64 * 70, max_entries=3 * 64 * 70 * 1024,
                     max_h=64, max_w=70, max_t=1024)
    synth = R.Context(64, 70, 1024, 2, irf.samples, irf.origin)
    payload = {}
    reqs = []
    for s, base in enumerate(bases):
        for k in range(5):
            sc = scenes.moving_frame(base, k)
            payload[(s, k)] = synth.synthesize(scenes.sampling_tables(sc))
            reqs.append(Request(s, k, base.h, base.w, base.t, arrival=0.0005 * k))
    for r in reqs:
        r.payload = payload[(r.stream, r.index)]
    be = GpuBackend(2, lim, irf.samples, irf.origin, prm, k_max=2, frame_source=None, depth_net=net)
    be.snapshots = {}
    be.results = {}
    srv = Server(be)
    done = srv.run(reqs, timeout_s=120)
    assert len(done) == len(reqs)
    assert max(len(b) for b in srv.batches) > 1          # frames were batched together
    alone = R.Context(64, 70, 1024, 2, irf.samples, irf.origin)
    if net is not None:
        alone.set_depth_net(net)
    for key, snap in be.snapshots.items():
        state = {k: v.clone() for k, v in snap["state"].items()}
        p = dict(prm, warm_start=1 if snap["warm"] else 0)
        alone.reconstruct(p, dense=snap["dense"], out=state)
        torch.cuda.synchronize()
        got, want = np_of(be.results[key]), np_of(state)
        for f in ("t", "r", "alive", "b", "n_points"):
            assert np.array_equal(np.asarray(got[f]), np.asarray(want[f])), (key, f)
