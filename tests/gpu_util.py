"""Helpers shared by the GPU parity tests: contexts, host/device conversion and
the oracle-vs-kernel comparison of point clouds."""
import numpy as np

import scenes


def torch_mod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def upload_u16(a):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).cuda().view(torch.uint16)


def u16_np(t):
    torch = torch_mod()
    return t.view(torch.int16).cpu().numpy().view(np.uint16)


def np_of(res):
    out = {}
    for k, v in res.items():
        if k == "n_points":
            out[k] = int(v.cpu().numpy()[0])
        else:
            out[k] = v.cpu().numpy()
    return out


def make_ctx(scene, k=None, max_batch=1, max_h=None, max_w=None, max_t=None, max_entries=0):
    from paper_1905_06700_b300 import rt3d as R
    k = k or max(1, scene.n_comp)
    return R.Context(max_h or scene.h, max_w or scene.w, max_t or scene.t, min(k, 4),
                     scene.irf.samples, scene.irf.origin, max_batch=max_batch,
                     max_entries=max_entries)


def oracle_irf(orc, scene):
    return orc.OIrf(scene.irf.samples, scene.irf.origin)


def state_to_device(st):
    torch = torch_mod()
    return dict(t=torch.from_numpy(st.t.astype(np.float32)).cuda(),
                r=torch.from_numpy(st.r.astype(np.float32)).cuda(),
                alive=torch.from_numpy(st.alive.copy()).cuda(),
                b=torch.from_numpy(st.b.astype(np.float32)).cuda(),
                n_points=torch.zeros(1, dtype=torch.int32).cuda())


def state_f32_rounded(orc, st):
    """The oracle state with every value rounded through float32 (the GPU's start)."""
    out = st.copy()
    out.t[:] = st.t.astype(np.float32)
    out.r[:] = st.r.astype(np.float32)
    out.b[:] = st.b.astype(np.float32)
    return out


def oracle_with_probes(orc, sc, z, prm, gain=None):
    """The FP64 oracle's reconstruction and its probe ensemble (oracle.compare):
    the same run with the state rounded after every step the way
    single-precision kernels round theirs."""
    from oracle import compare
    return compare.reconstruct_with_probes(z, oracle_irf(orc, sc), prm, gain=gain)


def compare_clouds(gpu, orc_state, T, tol_t=1e-3, tol_r=1e-4, probes=None, max_ill_frac=0.0,
                   label="", r_min=None, ratio=3.0):
    """Per point: the same alive set, depth within tol_t bins, intensity within
    tol_r relative (floor 0.1 photon); background within tol_r of the pixel's
    mean count rate b + sum r / T.  Points the probe ensemble marks
    ill-conditioned are held instead to the ensemble's own deviation
    (oracle.compare.cloud_stats): a flip only where a probe flips the point,
    an error within max(tolerance, ratio x the probes' deviation); their
    count is bounded by max_ill_frac of the points.  Backgrounds likewise: a
    pixel whose background a probe moves beyond half the tolerance is held to
    the ensemble's deviation, and such pixels are at most max_ill_frac of the
    pixels.  Returns statistics."""
    from oracle import compare
    st = compare.cloud_stats(gpu, orc_state, probes or [], T, tol_t, tol_r, r_min=r_min, ratio=ratio)
    n_pts = max(1, st["points"])
    assert st["ill"] <= max_ill_frac * n_pts, (label, "ill-conditioned", st)
    assert st["flips"] == 0, (label, st)
    assert st["dt_max"] <= tol_t, (label, st)
    assert st["dr_max"] <= tol_r, (label, st)
    assert st["db_max"] <= tol_r, (label, st)
    assert st["ill_flips_unexplained"] == 0, (label, st)
    assert st["ill_over_bound"] == 0, (label, st)
    assert st["ill_background_over_bound"] == 0, (label, st)
    assert st["ill_background_pixels"] <= max_ill_frac * orc_state.b.size, (label, "ill backgrounds", st)
    return st


def workload_params(scene, **over):
    return scenes.make_params(scene, **over)
