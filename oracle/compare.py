"""Comparison of a reconstruction with FP64 oracle runs (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this module.  It holds no arithmetic of the method: it runs the
oracle's own steps (oracle.py) and compares point clouds.

The method takes discontinuous decisions (pruning at r_min, the merge
distance, the denoisers' neighbour cut-offs) and has steep regions (photons
on the onset of a gamma IRF), so a perturbation of the size of single
precision rounding can move some points by far more than the rounding.  A
*probe* is the oracle's loop with its state rounded after every step the way
single-precision kernels perturb theirs: depths to `t_bits` significant bits
(24 = float32 storage; 23 and 25 stand for one more or one less rounding of
the depth arithmetic) and intensities and backgrounds to `rb_bits` (about the
rounding of a float32 sum of ~100 terms).  Points where the oracle and any
probe of the ensemble disagree beyond half the tolerance are ill-conditioned;
the GPU is held there to a bound set by the probes' own deviation
(cloud_stats).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

# the probe ensemble: (depth bits, intensity/background bits)
PROBE_BITS = ((24, 20), (24, 18), (23, 19), (25, 21), (24, 22))


def round_bits(a, bits):
    """Round every value to `bits` significant bits."""
    m, e = np.frexp(a)
    return np.ldexp(np.round(m * 2.0 ** bits) / 2.0 ** bits, e)


def _rnd(st, bits):
    t_bits, rb_bits = bits
    st.t[:] = st.t.astype(np.float32) if t_bits == 24 else round_bits(st.t, t_bits)
    st.r[:] = round_bits(st.r, rb_bits)
    st.b[:] = round_bits(st.b, rb_bits)


def probe_palm(fr, irf, prm, start, n_iter, bits):
    """The oracle's PALM loop from `start` (copied), rounded after every step
    (bits = (depth bits, intensity/background bits))."""
    st = start.copy()
    _rnd(st, bits)
    up = int(prm.get("upsample", 1))
    h, w, t = fr.hh, fr.ww, fr.tt
    for _ in range(n_iter):
        O.t_step(fr, irf, prm, st); _rnd(st, bits)
        O.depth_denoise(h * up, w * up, t, prm, st); _rnd(st, bits)
        O.r_step(fr, irf, prm, st); _rnd(st, bits)
        O.int_lowpass(h * up, w * up, prm, st); _rnd(st, bits)
        O.b_step(fr, irf, prm, st); _rnd(st, bits)
        O.bkg_lowpass(h, w, prm, st.b); _rnd(st, bits)
    return st


def reconstruct_with_probes(dense, irf, prm, gain=None, bits_list=PROBE_BITS, irf_idx=None):
    """(oracle reconstruction, [probe reconstructions]) of one frame."""
    o = O.reconstruct(dense, irf, prm, gain=gain, irf_idx=irf_idx)
    fr = O.OFrame(dense, gain, irf_idx)
    s0 = O.init(dense, gain, irf, prm, irf_idx=irf_idx)
    probes = [probe_palm(fr, irf, prm, s0, prm["n_iter"], b) for b in bits_list]
    return o, probes


def palm_with_probes(fr, irf, prm, start, n_iter, bits_list=PROBE_BITS):
    """(oracle loop, [probe loops]) from a given start state (warm starts)."""
    o = start.copy()
    O.palm(fr, irf, prm, o, n_iter)
    return o, [probe_palm(fr, irf, prm, start, n_iter, b) for b in bits_list]


def ill_mask(o, probe, tol_t, tol_r):
    """Points whose alive flag, depth (> tol_t/2) or intensity (> tol_r/2
    relative, floor 0.1 photon) differ between the oracle and one probe."""
    both = o.alive.astype(bool) & probe.alive.astype(bool)
    ill = o.alive != probe.alive
    ill |= both & (np.abs(o.t - probe.t) > 0.5 * tol_t)
    ill |= both & (np.abs(o.r - probe.r) > 0.5 * tol_r * np.maximum(np.abs(o.r), 0.1))
    return ill


def cloud_stats(gpu, o, probes, T, tol_t, tol_r, r_min=None, ratio=3.0):
    """Statistics of a reconstruction `gpu` (dict of numpy arrays t, r, alive,
    b) against the oracle state `o`, with the ill-conditioned points taken
    from the probe ensemble (a point is ill-conditioned if any probe moves it
    beyond half the tolerance, ill_mask).

    Well-conditioned points: flips (alive differs), depth error (bins),
    relative intensity error (floor 0.1 photon), background error relative to
    the pixel's mean count rate b + sum r / T (pixels without ill points whose
    background no probe moves beyond half the tolerance).

    Ill-conditioned points: each must satisfy, against the probe ensemble's
    envelope env = max over probes of |probe - oracle| (infinite where a probe
    flips the point):
      - a flip only where some probe flips the point too;
      - |t_gpu - t_o| <= max(tol_t, ratio * env_t) and the same for the
        relative intensity.
    `ill_ratio_max` is the largest |gpu - oracle| / env over the ill points
    whose error exceeds the tolerance (0 if none does).

    Backgrounds the same way: the background step is multiplicative in
    (b + eps) (Methods, background update), so a pixel whose background starts
    at the floor with photons its points do not explain grows it by orders of
    magnitude and amplifies rounding.  A pixel whose background some probe
    moves beyond half the tolerance, or that holds an ill point, is held to
    |b_gpu - b_o| / rate <= max(tol_r, ratio * env_b) (`ill_background_pixels`,
    `ill_background_over_bound`).

    Near-threshold points (the parity definition's exemption): oracle points
    whose final intensity lies within 1e-5 r_min of r_min (counted only)."""
    ga = gpu["alive"].astype(bool)
    oa = o.alive.astype(bool)
    ill = np.zeros_like(oa)
    for p in probes:
        ill |= ill_mask(o, p, tol_t, tol_r)
    ok = ~ill
    both = ga & oa
    dt_all = np.abs(gpu["t"].astype(np.float64) - o.t)
    rfl = np.maximum(np.abs(o.r), 0.1)
    dr_all = np.abs(gpu["r"].astype(np.float64) - o.r) / rfl
    well = both & ok
    # background: per pixel (with super-resolution the points sit on a finer
    # grid; a pixel's rate sums its block's points)
    up = o.t.shape[1] // o.b.shape[0]
    kk, hh, ww = o.t.shape
    blk = lambda a: a.reshape(kk, hh // up, up, ww // up, up).sum(axis=(0, 2, 4))
    ill_px = blk(ill.astype(np.int64)) > 0
    rate = np.maximum(o.b + blk(o.r * oa) / T, 1e-12)
    db_all = np.abs(gpu["b"].astype(np.float64) - o.b) / rate
    env_b = np.zeros_like(o.b)
    for p in probes:
        env_b = np.maximum(env_b, np.abs(p.b - o.b) / rate)
    ill_b = ill_px | (env_b > 0.5 * tol_r)
    db = db_all[~ill_b]
    b_over = ill_b & (db_all > np.maximum(tol_r, ratio * env_b))

    # envelope of the probes' own deviations
    env_t = np.zeros_like(o.t)
    env_r = np.zeros_like(o.r)
    probe_flip = np.zeros_like(oa)
    for p in probes:
        pa = p.alive.astype(bool)
        probe_flip |= pa != oa
        env_t = np.maximum(env_t, np.where(pa & oa, np.abs(p.t - o.t), 0.0))
        env_r = np.maximum(env_r, np.where(pa & oa, np.abs(p.r - o.r) / rfl, 0.0))
    env_t = np.where(probe_flip, np.inf, env_t)
    env_r = np.where(probe_flip, np.inf, env_r)
    ill_flips = ill & (ga != oa)
    ill_flip_unexplained = ill_flips & ~probe_flip
    ib = ill & both
    bound_t = np.maximum(tol_t, ratio * env_t)
    bound_r = np.maximum(tol_r, ratio * env_r)
    ill_over = ib & ((dt_all > bound_t) | (dr_all > bound_r))
    with np.errstate(divide="ignore", invalid="ignore"):
        rt = np.where(ib & (dt_all > tol_t), dt_all / env_t, 0.0)
        rr = np.where(ib & (dr_all > tol_r), dr_all / env_r, 0.0)
    rt = np.nan_to_num(rt, nan=np.inf, posinf=np.inf)
    rr = np.nan_to_num(rr, nan=np.inf, posinf=np.inf)
    dtw = dt_all[well]
    dta = dt_all[both]
    st = dict(points=int(oa.sum()), ill=int(ill.sum()),
              flips=int(((ga != oa) & ok).sum()),
              dt_max=float(dtw.max()) if dtw.size else 0.0,
              dt_p999=float(np.percentile(dtw, 99.9)) if dtw.size else 0.0,
              dr_max=float(dr_all[well].max()) if well.any() else 0.0,
              db_max=float(db.max()) if db.size else 0.0,
              ill_background_pixels=int((ill_b & ~ill_px).sum()),
              ill_background_over_bound=int(b_over.sum()),
              ill_flips=int(ill_flips.sum()),
              ill_flips_unexplained=int(ill_flip_unexplained.sum()),
              ill_over_bound=int(ill_over.sum()),
              ill_ratio_max=float(max(rt.max(initial=0.0), rr.max(initial=0.0))),
              ill_dt_max=float(dt_all[ib].max()) if ib.any() else 0.0,
              all_dt_max=float(dta.max()) if dta.size else 0.0,
              all_dt_p999=float(np.percentile(dta, 99.9)) if dta.size else 0.0,
              all_frac_within_tol=float((dta <= tol_t).mean()) if dta.size else 1.0,
              all_alive_mismatch=int((ga != oa).sum()))
    if r_min is not None:
        near = oa & (np.abs(o.r - r_min) <= 1e-5 * r_min)
        st["near_threshold"] = int(near.sum())
    return st
