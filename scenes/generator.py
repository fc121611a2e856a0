"""Scene recipes and photon-sampling tables.

A scene gives, per pixel (i, j) and per surface component s:
  * the true depth d_s(i, j) in histogram bins (NaN where the component is absent),
  * the expected number of signal photons mu_s(i, j) it returns,
and per pixel the expected background photons per bin b(i, j), plus one
instrument response (IRF) sampled at integer bin offsets.

Photon synthesis (done independently by the oracle and by the CUDA library)
turns these into a histogram with integer operations only, driven by the
Philox4x32-10 counter-based generator.  This module supplies the integer
tables those samplers need:

  * Poisson counts: a mean mu is split into m = ceil(mu / 16) equal parts; each
    part is drawn by fixed-point inversion from p0 = round(exp(-mu/m) * 2^62)
    and MU = round(mu/m * 2^32).
  * Photon time offsets: the IRF's cumulative distribution as uint32
    thresholds (an offset index is the number of thresholds <= a uniform word).
  * Sub-bin depth: a photon lands one bin later with probability frac(d),
    encoded as the uint32 threshold floor(frac(d) * 2^32).

The expected histogram of pixel p is therefore
    E z_t = b * T * (1/T) + sum_s mu_s [(1 - f_s) pi(t - floor(d_s) + o)
                                        + f_s pi(t - floor(d_s) - 1 + o)]
with pi the quantised IRF probabilities and o the IRF origin, i.e. the
likelihood's mean with a linearly interpolated sub-bin shift.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BG_COMPONENT = 255          # Philox component index used for background photons
POISSON_PART_MAX = 16.0     # largest mean handled by one fixed-point inversion


@dataclasses.dataclass
class Irf:
    samples: np.ndarray     # float64 [L], unnormalised, h_k at offset k - origin
    origin: int             # sample index that sits at depth offset 0

    @property
    def length(self) -> int:
        return int(self.samples.shape[0])

    def normalised(self) -> np.ndarray:
        return self.samples / self.samples.sum()

    def fisher_information(self) -> float:
        """Location Fisher information sum h'^2 / h of the normalised samples
        (central differences), i.e. 1/sigma^2 for a Gaussian pulse."""
        h = self.normalised()
        d = np.gradient(h)
        m = h > 1e-6 * h.max()
        return float((d[m] ** 2 / h[m]).sum())

    def variance(self) -> float:
        h = self.normalised()
        k = np.arange(self.length) - self.origin
        m = float((h * k).sum())
        return float((h * (k - m) ** 2).sum())


@dataclasses.dataclass
class Scene:
    h: int
    w: int
    t: int
    depth: np.ndarray        # float64 [S][H][W]; NaN = component absent
    signal: np.ndarray       # float64 [S][H][W]; expected signal photons
    bkg: np.ndarray          # float64 [H][W]; expected background photons per bin
    irf: Irf
    seed: int                # Philox key for the photon draws
    name: str = "scene"

    @property
    def n_comp(self) -> int:
        return int(self.depth.shape[0])


def gaussian_irf(sigma: float = 4.0, half: int = 16) -> Irf:
    """Gaussian pulse sampled at integer offsets -half..half; origin at the peak."""
    k = np.arange(-half, half + 1, dtype=np.float64)
    return Irf(np.exp(-0.5 * (k / sigma) ** 2), half)


def gamma_irf(shape: float = 3.0, scale: float = 5.0, length: int = 80) -> Irf:
    """Gamma-shaped pulse sampled at bin centres on [0, length); origin = argmax,
    so that a depth names the position of the pulse peak."""
    x = np.arange(length, dtype=np.float64) + 0.5
    h = x ** (shape - 1.0) * np.exp(-x / scale)
    return Irf(h, int(np.argmax(h)))


# ---------------------------------------------------------------------------
# integer sampling tables
# ---------------------------------------------------------------------------

def _poisson_fixed(mu: np.ndarray):
    """Per-entry (n_parts, p0, MU) of the fixed-point Poisson sampler."""
    mu = np.asarray(mu, dtype=np.float64)
    mu = np.where(np.isfinite(mu) & (mu > 0), mu, 0.0)
    parts = np.where(mu > 0, np.ceil(mu / POISSON_PART_MAX), 0).astype(np.uint32)
    per = np.where(parts > 0, mu / np.maximum(parts, 1), 0.0)
    p0 = np.where(parts > 0, np.rint(np.exp(-per) * 2.0 ** 62), 0).astype(np.uint64)
    mu_fx = np.where(parts > 0, np.rint(per * 2.0 ** 32), 0).astype(np.uint64)
    return parts, p0, mu_fx


def irf_cdf_thresholds(irf: Irf) -> np.ndarray:
    """uint32 thresholds C_0..C_{L-2}: offset index = #{s : C_s <= u}."""
    h = irf.normalised()
    c = np.cumsum(h)[:-1]
    thr = np.floor(c * 2.0 ** 32)
    return np.minimum(thr, 2.0 ** 32 - 1).astype(np.uint32)


def sampling_tables(scene: Scene) -> dict:
    """All integer inputs of the photon samplers for one scene."""
    s, h, w = scene.depth.shape
    present = np.isfinite(scene.depth) & (scene.signal > 0)
    d = np.where(present, scene.depth, 0.0)
    d_int = np.floor(d)
    frac = d - d_int
    split = np.minimum(np.floor(frac * 2.0 ** 32), 2.0 ** 32 - 1).astype(np.uint32)
    mu = np.zeros((s + 1, h, w))
    mu[:s] = np.where(present, scene.signal, 0.0)
    mu[s] = scene.bkg * scene.t
    parts, p0, mu_fx = _poisson_fixed(mu)
    return dict(
        h=h, w=w, t=scene.t, n_comp=s, seed=int(scene.seed),
        depth_int=np.ascontiguousarray(d_int.astype(np.int32)),
        depth_split=np.ascontiguousarray(split),
        n_parts=np.ascontiguousarray(parts),
        p0=np.ascontiguousarray(p0),
        mu=np.ascontiguousarray(mu_fx),
        irf_cdf=np.ascontiguousarray(irf_cdf_thresholds(scene.irf)),
        irf_len=scene.irf.length, irf_origin=int(scene.irf.origin),
    )


def quantised_irf_pmf(irf: Irf) -> np.ndarray:
    """Probabilities of each offset index under the uint32 thresholds."""
    thr = irf_cdf_thresholds(irf).astype(np.float64)
    edges = np.concatenate([[0.0], thr, [2.0 ** 32]])
    return np.diff(edges) / 2.0 ** 32


def expected_histogram(scene: Scene) -> np.ndarray:
    """E z [H][W][T] of the sampler defined above (photons outside [0, T) are lost)."""
    tab = sampling_tables(scene)
    pmf = quantised_irf_pmf(scene.irf)
    o = scene.irf.origin
    out = np.repeat(scene.bkg[:, :, None], scene.t, axis=2).astype(np.float64)
    split = tab["depth_split"].astype(np.float64) / 2.0 ** 32
    for s in range(scene.n_comp):
        mu = np.where(np.isfinite(scene.depth[s]) & (scene.signal[s] > 0), scene.signal[s], 0.0)
        for i in range(scene.h):
            for j in range(scene.w):
                if mu[i, j] <= 0:
                    continue
                base = int(tab["depth_int"][s, i, j]) - o
                f = split[s, i, j]
                for k, p in enumerate(pmf):
                    for shift, wgt in ((0, 1.0 - f), (1, f)):
                        tb = base + k + shift
                        if 0 <= tb < scene.t:
                            out[i, j, tb] += mu[i, j] * p * wgt
    return out


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def _reflectivity(rng, shape, mean_photons):
    refl = rng.uniform(0.2, 1.0, size=shape)
    return refl * (mean_photons / refl.mean())


def plane_hemisphere(h=32, w=32, t=1024, seed=1, mean_signal=10.0, bkg=0.01,
                     pitch=16.0) -> Scene:
    """One surface per pixel: a tilted plane with a hemisphere bulging towards
    the sensor; depths within bins 200-800 (for the default 32x32x1024)."""
    rng = np.random.default_rng(seed)
    i, j = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64),
                       indexing="ij")
    depth = 250.0 + 500.0 * (0.6 * i / max(h - 1, 1) + 0.4 * j / max(w - 1, 1))
    ci, cj, rad = 0.40 * (h - 1), 0.60 * (w - 1), 0.25 * min(h, w)
    rho2 = (i - ci) ** 2 + (j - cj) ** 2
    bulge = np.where(rho2 < rad ** 2, np.sqrt(np.maximum(rad ** 2 - rho2, 0.0)) * pitch, 0.0)
    depth = depth - 0.5 * bulge
    depth = depth * (t / 1024.0)
    sig = _reflectivity(rng, (h, w), mean_signal)
    return Scene(h, w, t, depth[None], sig[None], np.full((h, w), bkg), gaussian_irf(4.0, 16),
                 seed, "plane_hemisphere")


def net_object_wall(h=141, w=141, t=4096, seed=1, mean_signal=5.0, sbr=1.0,
                    irf: Irf | None = None) -> Scene:
    """Up to three surfaces per pixel: a camouflage-like net at bin 1500 (strands
    2 px wide every 12 px, ~31 % fill, half of the light on net pixels), a smooth
    ellipsoidal object spanning bins 1800-2200 and a wall at bin 3000 behind it;
    object-edge pixels split their remaining light between object and wall."""
    irf = irf or gamma_irf(3.0, 5.0, 80)
    rng = np.random.default_rng(seed)
    sc = t / 4096.0
    i, j = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64),
                       indexing="ij")
    net = ((np.arange(h)[:, None] % 12) < 2) | ((np.arange(w)[None, :] % 12) < 2)
    ci, cj = 0.5 * (h - 1), 0.5 * (w - 1)
    ai, aj = 0.33 * h, 0.25 * w
    rho = np.sqrt(((i - ci) / ai) ** 2 + ((j - cj) / aj) ** 2)
    inside = rho < 1.0
    edge = inside & (rho > 0.9)
    obj_depth = (2200.0 - 400.0 * np.sqrt(np.maximum(1.0 - rho ** 2, 0.0))) * sc
    total = _reflectivity(rng, (h, w), mean_signal)
    behind = np.where(net, 0.5, 1.0) * total
    depth = np.full((3, h, w), np.nan)
    sig = np.zeros((3, h, w))
    depth[0] = np.where(net, 1500.0 * sc, np.nan)
    sig[0] = np.where(net, 0.5 * total, 0.0)
    depth[1] = np.where(inside, obj_depth, np.nan)
    sig[1] = np.where(inside, np.where(edge, 0.5, 1.0) * behind, 0.0)
    depth[2] = np.where(~inside | edge, 3000.0 * sc, np.nan)
    sig[2] = np.where(~inside, behind, np.where(edge, 0.5 * behind, 0.0))
    bkg = np.full((h, w), mean_signal / sbr / t)
    return Scene(h, w, t, depth, sig, bkg, irf, seed, "net_object_wall")


def two_layer(h=256, w=256, t=4096, seed=1, mean_signal=5.0, sbr=0.1) -> Scene:
    """Two surfaces per pixel: a semi-transparent tilted layer near bin 1500
    carrying 40 % of the light, and behind it the ellipsoidal object or the wall."""
    irf = gamma_irf(3.0, 5.0, 80)
    rng = np.random.default_rng(seed)
    sc = t / 4096.0
    i, j = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64),
                       indexing="ij")
    ci, cj = 0.5 * (h - 1), 0.5 * (w - 1)
    rho = np.sqrt(((i - ci) / (0.33 * h)) ** 2 + ((j - cj) / (0.25 * w)) ** 2)
    inside = rho < 1.0
    total = _reflectivity(rng, (h, w), mean_signal)
    depth = np.empty((2, h, w))
    sig = np.empty((2, h, w))
    depth[0] = (1400.0 + 200.0 * (i + j) / max(h + w - 2, 1)) * sc
    sig[0] = 0.4 * total
    depth[1] = np.where(inside, 2200.0 - 400.0 * np.sqrt(np.maximum(1 - rho ** 2, 0)), 3000.0) * sc
    sig[1] = 0.6 * total
    bkg = np.full((h, w), mean_signal / sbr / t)
    return Scene(h, w, t, depth, sig, bkg, irf, seed, "two_layer")


def head_like(h=141, w=141, t=4096, seed=1, mean_signal=3.0, bkg_photons=1.0) -> Scene:
    """The shape of the paper's raster-scan head frame (141 x 141 pixels, a few
    signal photons per pixel, mostly one surface per pixel and two at the
    head's border): an ellipsoidal head in front of a back plane, its rim
    pixels splitting their light between the two; gamma IRF (3, 5);
    mean_signal signal photons and bkg_photons background photons per pixel
    (uniform over the T bins).  Used for the execution-time sweeps of Fig. 5
    (pixel count, mean active bins per pixel)."""
    irf = gamma_irf(3.0, 5.0, 80)
    rng = np.random.default_rng(seed)
    sc = t / 4096.0
    i, j = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    rho = np.sqrt(((i - 0.5 * (h - 1)) / (0.36 * h)) ** 2 + ((j - 0.5 * (w - 1)) / (0.27 * w)) ** 2)
    inside = rho < 1.0
    rim = inside & (rho > 0.92)
    total = _reflectivity(rng, (h, w), mean_signal)
    depth = np.full((2, h, w), np.nan)
    sig = np.zeros((2, h, w))
    depth[0] = np.where(inside, (2000.0 - 300.0 * np.sqrt(np.maximum(1.0 - rho ** 2, 0.0))) * sc, np.nan)
    sig[0] = np.where(inside, np.where(rim, 0.5, 1.0) * total, 0.0)
    depth[1] = np.where(~inside | rim, (2600.0 + 0.5 * (i - h / 2)) * sc, np.nan)
    sig[1] = np.where(~inside, total, np.where(rim, 0.5 * total, 0.0))
    bkg = np.full((h, w), bkg_photons / t)
    return Scene(h, w, t, depth, sig, bkg, irf, seed, "head_like")


def super_resolved(world_depth: np.ndarray, world_signal: np.ndarray, bkg: np.ndarray, t: int, irf: Irf,
                   up: int, seed: int, name: str = "super_resolved") -> Scene:
    """A lidar frame observing a world-resolution scene through the point-to-
    cube mapping f of Results, "Observation model", with super-resolution:
    each lidar pixel (i, j) sees the u x u world pixels (u i + a, u j + c).
    world_depth / world_signal are [S][u h][u w] (NaN / 0 where a surface is
    absent); sub-pixel a u + c and surface s become component (a u + c) S + s
    of the lidar pixel, so the sampler draws each world point's photons."""
    S, hu, wu = world_depth.shape
    h, w = hu // up, wu // up
    depth = np.full((up * up * S, h, w), np.nan)
    sig = np.zeros((up * up * S, h, w))
    for a in range(up * up):
        ai, aj = divmod(a, up)
        for s in range(S):
            depth[a * S + s] = world_depth[s, ai::up, aj::up]
            sig[a * S + s] = world_signal[s, ai::up, aj::up]
    return Scene(h, w, t, depth, sig, np.asarray(bkg, np.float64), irf, seed, name)


def camouflage_people(h=32, w=32, t=153, up=3, seed=1, signal=450.0, bkg_photons=450.0, frame=0):
    """The paper's dynamic-scene shape (Results, "3D Dynamic scenes"): a
    32 x 32-pixel array with T = 153 bins observing, on a 3x finer world grid,
    a camouflage net in front, two people walking behind it and a backplane;
    about 450 signal and 450 background photons per pixel.  Most world pixels
    see two surfaces (the net's holes show one), and a lidar pixel on a
    person's contour mixes up to three depths.  Returns (scene, world_depth
    [2][u h][u w]).  `frame` moves the people 1 world pixel sideways per frame."""
    rng = np.random.default_rng(seed)
    hu, wu = h * up, w * up
    i, j = np.meshgrid(np.arange(hu, dtype=np.float64), np.arange(wu, dtype=np.float64), indexing="ij")
    # the net: a smooth random field thresholded to ~55 % cover
    field = np.zeros((hu, wu))
    for _ in range(6):
        fi, fj, ph = rng.uniform(0.15, 0.5), rng.uniform(0.15, 0.5), rng.uniform(0, 2 * np.pi)
        field += np.sin(fi * i + ph) * np.cos(fj * j + 0.7 * ph)
    net = field > np.quantile(field, 0.45)
    net_depth = 0.30 * t + 0.02 * t * (j / wu)
    # two people: upright ellipses with a head, at different depths
    person = np.zeros((hu, wu), bool)
    p_depth = np.full((hu, wu), np.nan)
    for cx, d0, ww_ in ((0.33 * wu + frame, 0.55 * t, 0.09 * wu), (0.68 * wu - frame, 0.60 * t, 0.08 * wu)):
        body = (((j - cx) / ww_) ** 2 + ((i - 0.62 * hu) / (0.30 * hu)) ** 2) < 1.0
        head = ((j - cx) ** 2 + (i - 0.25 * hu) ** 2) < (0.45 * ww_) ** 2
        m = (body | head) & ~person
        p_depth = np.where(m, d0 - 2.0 * np.sqrt(np.maximum(1.0 - ((j - cx) / ww_) ** 2, 0.0)), p_depth)
        person |= m
    wall_depth = 0.78 * t + 0.01 * t * (i / hu)
    depth = np.full((2, hu, wu), np.nan)
    sig = np.zeros((2, hu, wu))
    per_world = signal / (up * up)
    refl = rng.uniform(0.6, 1.0, (hu, wu))
    refl *= 1.0 / refl.mean()
    depth[0] = np.where(net, net_depth, np.nan)
    sig[0] = np.where(net, 0.4 * per_world * refl, 0.0)
    depth[1] = np.where(person, p_depth, wall_depth)
    sig[1] = np.where(net, 0.6, 1.0) * per_world * refl
    irf = gaussian_irf(1.0, 4)
    sc = super_resolved(depth, sig, np.full((h, w), bkg_photons / t), t, irf, up,
                        seed * 1_000_003 + frame, "camouflage_people")
    return sc, depth


def random_shapes(h=256, w=256, t=2048, seed=0) -> Scene:
    """Random planes, spheres and boxes (at most two surfaces per pixel), with
    1-20 signal photons per pixel and a signal-to-background ratio in 0.05-2."""
    rng = np.random.default_rng(seed)
    i, j = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64),
                       indexing="ij")
    back = (0.6 + 0.3 * rng.random()) * t + rng.uniform(-0.5, 0.5) * (i - h / 2) \
        + rng.uniform(-0.5, 0.5) * (j - w / 2)
    front = np.full((h, w), np.nan)
    for _ in range(rng.integers(1, 4)):
        kind = rng.integers(0, 3)
        ci, cj = rng.uniform(0.2, 0.8) * h, rng.uniform(0.2, 0.8) * w
        rad = rng.uniform(0.1, 0.3) * min(h, w)
        base = rng.uniform(0.2, 0.5) * t
        if kind == 0:       # sphere cap
            rho2 = (i - ci) ** 2 + (j - cj) ** 2
            m = rho2 < rad ** 2
            d = base - 4.0 * np.sqrt(np.maximum(rad ** 2 - rho2, 0))
        elif kind == 1:     # box face
            m = (np.abs(i - ci) < rad) & (np.abs(j - cj) < 0.7 * rad)
            d = np.full((h, w), base)
        else:               # tilted plane patch
            m = (np.abs(i - ci) < rad) & (np.abs(j - cj) < rad)
            d = base + rng.uniform(-2, 2) * (i - ci) + rng.uniform(-2, 2) * (j - cj)
        front = np.where(m & ~np.isfinite(front), d, front)
    front = np.clip(front, 100, t - 100)
    back = np.clip(back, 100, t - 100)
    photons = rng.uniform(1, 20)
    sbr = rng.uniform(0.05, 2.0)
    total = _reflectivity(rng, (h, w), photons)
    has_front = np.isfinite(front)
    share = rng.uniform(0.3, 0.7)
    depth = np.stack([front, back])
    sig = np.stack([np.where(has_front, share * total, 0.0),
                    np.where(has_front, (1 - share) * total, total)])
    bkg = np.full((h, w), photons / sbr / t)
    return Scene(h, w, t, depth, sig, bkg, gaussian_irf(3.0, 12), seed + 100_000, "random_shapes")


def small_random(h, w, t, n_comp=2, seed=0, mean_signal=20.0, bkg=0.005,
                 irf: Irf | None = None, pitch=16.0) -> Scene:
    """Small smooth multi-surface scene for parity tests of ragged shapes."""
    irf = irf or gaussian_irf(3.0, 12)
    rng = np.random.default_rng(seed)
    i, j = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64),
                       indexing="ij")
    depth = np.full((n_comp, h, w), np.nan)
    sig = np.zeros((n_comp, h, w))
    lo, hi = 40.0, t - 40.0
    for s in range(n_comp):
        c0 = lo + (s + 0.5) * (hi - lo) / n_comp
        gi, gj = rng.uniform(-0.3, 0.3, size=2) * pitch
        curv = rng.uniform(-0.05, 0.05)
        d = c0 + gi * (i - h / 2) / 4 + gj * (j - w / 2) / 4 + curv * ((i - h / 2) ** 2 + (j - w / 2) ** 2)
        d = np.clip(d, lo, hi)
        cover = rng.random((h, w)) < (1.0 if s == 0 else 0.7)
        depth[s] = np.where(cover, d, np.nan)
        sig[s] = np.where(cover, rng.uniform(0.5, 1.5, size=(h, w)) * mean_signal, 0.0)
    return Scene(h, w, t, depth, sig, np.full((h, w), bkg), irf, seed + 7, "small_random")


def moving_frame(base: Scene, frame: int, speed: float = 1.0) -> Scene:
    """The same scene translated in depth by speed * frame bins (a moving stream)."""
    return dataclasses.replace(base, depth=base.depth + speed * frame,
                               seed=base.seed * 1_000_003 + frame)


# ---------------------------------------------------------------------------
# reconstruction parameters per workload (plain numbers)
# ---------------------------------------------------------------------------

def make_params(scene: Scene, **over) -> dict:
    """Default reconstruction parameters for a workload.  The depth step is half
    a Fisher-scoring step (t_step = 0.5 / I_h), clamped to one IRF standard
    deviation; the APSS radius is 3.5 pixels in world units
    (7x7 pixel window)."""
    var = scene.irf.variance()
    pitch = over.pop("pixel_pitch", 16.0)
    p = dict(
        n_iter=20, k_max=max(1, scene.n_comp),
        t_step=0.5 / scene.irf.fisher_information(), r_step=0.5, b_step=0.5,
        dt_max=math.sqrt(var), eps_r=1e-3, eps_b=1e-6, b_floor=1e-7, lam_floor=1e-9,
        pixel_pitch=pitch, apss_radius=3.5 * pitch, win_r=3, apss_min_nb=6,
        int_radius=3.5 * pitch, r_min=0.5, merge_dist=max(2.0, 2.0 * math.sqrt(var)),
        depth_denoiser=1, intensity_denoiser=1, bkg_mode=0, bkg_sigma=1.0, bkg_radius=3,
        lmf_delta_rel=1e-3, lmf_frac_bits=5, peak_min_photons=2,
        peak_sep=max(2, int(math.ceil(2.0 * math.sqrt(var)))),
        lmf_precision=0, warm_start=0,
        net_scale=math.sqrt(var), net_fallback=math.sqrt(var) / 3.0, apss_fp64=0, upsample=1,
    )
    p.update(over)
    return p
