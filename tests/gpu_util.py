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


def _round_bits(a, bits):
    """Round every value to `bits` significant bits (a perturbation probe)."""
    m, e = np.frexp(a)
    return np.ldexp(np.round(m * 2.0 ** bits) / 2.0 ** bits, e)


def oracle_with_probe(orc, sc, z, prm, gain=None, bits=20):
    """The FP64 oracle's reconstruction, plus the same run perturbed after every
    step the way single-precision kernels perturb it: depths rounded to float32
    (the kernels store them so), intensities and backgrounds to `bits`
    significant bits (about the rounding of a float32 sum of ~100 terms).
    Points where the two runs differ are ill-conditioned: the method itself
    moves them under a perturbation of that size, so no FP32 implementation
    can be held to the oracle there."""
    irf = oracle_irf(orc, sc)
    a = orc.reconstruct(z, irf, prm, gain=gain)
    fr = orc.OFrame(z, gain)
    b = orc.init(z, gain, irf, prm)

    def rnd(s):
        s.t[:] = s.t.astype(np.float32)
        s.r[:] = _round_bits(s.r, bits)
        s.b[:] = _round_bits(s.b, bits)
    rnd(b)
    for _ in range(prm["n_iter"]):
        orc.t_step(fr, irf, prm, b); rnd(b)
        if prm["depth_denoiser"] == 1:
            orc.apss(sc.h, sc.w, sc.t, prm, b); rnd(b)
        orc.r_step(fr, irf, prm, b); rnd(b)
        orc.int_lowpass(sc.h, sc.w, prm, b); rnd(b)
        orc.b_step(fr, irf, prm, b); rnd(b)
        orc.bkg_lowpass(sc.h, sc.w, prm, b.b); rnd(b)
    return a, b


def ill_conditioned(a, b, tol_t, tol_r):
    """Points whose alive flag, depth (> tol_t/2) or intensity (> tol_r/2 relative)
    differ between the oracle run and its perturbed twin."""
    both = a.alive.astype(bool) & b.alive.astype(bool)
    ill = a.alive != b.alive
    ill |= both & (np.abs(a.t - b.t) > 0.5 * tol_t)
    ill |= both & (np.abs(a.r - b.r) > 0.5 * tol_r * np.maximum(np.abs(a.r), 0.1))
    return ill


def compare_clouds(gpu, orc_state, T, tol_t=1e-3, tol_r=1e-4, ill=None, max_ill_frac=0.0,
                   label=""):
    """Per point: the same alive set, depth within tol_t bins, intensity within
    tol_r relative (floor 0.1 photon); background within tol_r of the pixel's
    mean count rate b + sum r / T.  Points flagged ill-conditioned by the
    oracle's perturbation probe are excluded (their count is bounded by
    max_ill_frac of the points).  Returns statistics."""
    ga = gpu["alive"].astype(bool)
    oa = orc_state.alive.astype(bool)
    K, H, W = ga.shape
    ill = np.zeros_like(ga) if ill is None else ill.astype(bool)
    n_pts = max(1, int(oa.sum()))
    assert ill.sum() <= max_ill_frac * n_pts, (label, "ill-conditioned", int(ill.sum()), n_pts)
    ill_px = ill.any(0)
    ok = ~ill
    flips = (ga != oa) & ok
    both = ga & oa & ok
    dt = np.abs(gpu["t"].astype(np.float64) - orc_state.t)[both]
    dr = (np.abs(gpu["r"].astype(np.float64) - orc_state.r) /
          np.maximum(np.abs(orc_state.r), 0.1))[both]
    rate = orc_state.b + (orc_state.r * oa).sum(0) / T
    db = (np.abs(gpu["b"].astype(np.float64) - orc_state.b) / np.maximum(rate, 1e-12))[~ill_px]
    stats = dict(points=n_pts, ill=int(ill.sum()), flips=int(flips.sum()),
                 dt_max=float(dt.max()) if dt.size else 0.0,
                 dt_p999=float(np.percentile(dt, 99.9)) if dt.size else 0.0,
                 dr_max=float(dr.max()) if dr.size else 0.0,
                 db_max=float(db.max()) if db.size else 0.0)
    assert stats["flips"] == 0, (label, stats)
    assert stats["dt_max"] <= tol_t, (label, stats)
    assert stats["dr_max"] <= tol_r, (label, stats)
    assert stats["db_max"] <= tol_r, (label, stats)
    return stats


def workload_params(scene, **over):
    return scenes.make_params(scene, **over)
