"""ctypes wrapper of the FP64 C oracle (test infrastructure only).

The C sources beside this file implement, in plain loops, the observation
model, the log-matched-filter initialisation and the PALM iteration with its
denoisers (see rt3d_oracle.h for the paper passages).  This wrapper only
builds the library, compacts histograms into per-pixel nonzero-bin lists and
marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "build", "liboracle.so")
SOURCES = ["synth.c", "model.c", "init.c", "denoise.c", "palm.c", "net.c"]

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over pixels) if it is out of date."""
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "rt3d_oracle.h")]
    if not force and os.path.exists(LIB_PATH):
        built = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(d) <= built for d in deps):
            return LIB_PATH
    os.makedirs(os.path.dirname(LIB_PATH), exist_ok=True)
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
           "-Wno-unknown-pragmas", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Irf(C.Structure):
    _fields_ = [("len", C.c_int), ("origin", C.c_int), ("h", C.POINTER(C.c_double))]


class Frame(C.Structure):
    _fields_ = [("h", C.c_int), ("w", C.c_int), ("t", C.c_int),
                ("off", C.POINTER(C.c_int64)), ("bin", C.POINTER(C.c_int32)),
                ("cnt", C.POINTER(C.c_double)), ("gain", C.POINTER(C.c_double)),
                ("irf_idx", C.POINTER(C.c_uint8))]


class State(C.Structure):
    _fields_ = [("k", C.c_int), ("t", C.POINTER(C.c_double)), ("r", C.POINTER(C.c_double)),
                ("alive", C.POINTER(C.c_uint8)), ("b", C.POINTER(C.c_double))]


class Params(C.Structure):
    _fields_ = [("n_iter", C.c_int), ("k_max", C.c_int),
                ("t_step", C.c_double), ("r_step", C.c_double), ("b_step", C.c_double),
                ("dt_max", C.c_double), ("eps_r", C.c_double), ("eps_b", C.c_double),
                ("b_floor", C.c_double), ("lam_floor", C.c_double),
                ("pixel_pitch", C.c_double), ("apss_radius", C.c_double),
                ("win_r", C.c_int), ("apss_min_nb", C.c_int),
                ("int_radius", C.c_double), ("r_min", C.c_double), ("merge_dist", C.c_double),
                ("depth_denoiser", C.c_int), ("intensity_denoiser", C.c_int),
                ("bkg_mode", C.c_int), ("bkg_sigma", C.c_double), ("bkg_radius", C.c_int),
                ("lmf_delta_rel", C.c_double), ("lmf_frac_bits", C.c_int),
                ("peak_min_photons", C.c_int), ("peak_sep", C.c_int),
                ("net_theta", C.POINTER(C.c_double)), ("net_scale", C.c_double),
                ("net_fallback", C.c_double), ("upsample", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.or_poisson_fixed.restype = C.c_uint32
        _lib.or_nll_dense.restype = C.c_double
        _lib.or_nll_dense_idx.restype = C.c_double
        _lib.or_peaks.restype = C.c_int
        _lib.or_num_threads.restype = C.c_int
        _lib.or_net_nparams.restype = C.c_long
        _lib.or_net_offset.restype = C.c_long
        _lib.or_net_cin.restype = C.c_int
        _lib.or_net_cout.restype = C.c_int
        _lib.or_bf16.restype = C.c_double
        _lib.or_bf16.argtypes = [C.c_double]
        _lib.or_net_loss.restype = C.c_double
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _f32(v):
    """Parameters are rounded to single precision, the precision the kernels see."""
    return float(np.float32(v))


def make_params(d: dict) -> Params:
    """Oracle parameters from a parameter dict; floats pass through float32 so
    that both sides see the same constants.  The learned denoiser's parameter
    vector, if any, is d["net_theta"] (float64 array, kept alive by the
    returned object)."""
    p = Params()
    for name, ctype in Params._fields_:
        if name == "net_theta":
            th = d.get("net_theta")
            if th is not None:
                th = np.ascontiguousarray(th, np.float64)
                p._theta = th
                p.net_theta = th.ctypes.data_as(C.POINTER(C.c_double))
            continue
        if name in ("net_scale", "net_fallback") and name not in d:
            v = 1.0
        elif name == "upsample" and name not in d:
            v = 1
        else:
            v = d[name]
        setattr(p, name, int(v) if ctype is C.c_int else _f32(v))
    return p


@dataclasses.dataclass
class OState:
    t: np.ndarray      # float64 [K][H][W]
    r: np.ndarray
    alive: np.ndarray  # uint8 [K][H][W]
    b: np.ndarray      # float64 [H][W]

    def copy(self):
        return OState(self.t.copy(), self.r.copy(), self.alive.copy(), self.b.copy())

    def c(self):
        return State(self.t.shape[0], _ptr(self.t, C.c_double), _ptr(self.r, C.c_double),
                     _ptr(self.alive, C.c_uint8), _ptr(self.b, C.c_double))


def new_state(k, h, w, up=1) -> OState:
    """A state for an h x w frame: points on the world grid (up times finer
    with super-resolution), the background per pixel."""
    hh, ww = h * up, w * up
    return OState(np.zeros((k, hh, ww)), np.zeros((k, hh, ww)), np.zeros((k, hh, ww), np.uint8),
                  np.zeros((h, w)))


class OIrf:
    """IRF normalised in FP64 by the oracle (sum of samples in index order)."""

    def __init__(self, samples, origin):
        s = np.asarray(samples, dtype=np.float64)
        total = 0.0
        for v in s:
            total += float(v)
        self.h = np.ascontiguousarray(s / total)
        self.origin = int(origin)

    def c(self):
        return Irf(len(self.h), self.origin, _ptr(self.h, C.c_double))


def _irfs(irf):
    """An OIrf, or a list of them (the per-pixel responses a frame's irf_idx
    selects from), as the C array the oracle takes."""
    lst = list(irf) if isinstance(irf, (list, tuple)) else [irf]
    arr = (Irf * len(lst))(*[i.c() for i in lst])
    arr._keep = lst
    return arr


class OFrame:
    """Per-pixel nonzero-bin lists of a histogram (integer or expected counts),
    with an optional per-pixel index into a list of IRFs."""

    def __init__(self, z, gain=None, irf_idx=None):
        z = np.asarray(z)
        self.hh, self.ww, self.tt = z.shape
        flat = z.reshape(-1, self.tt)
        rows, bins = np.nonzero(flat)
        counts = np.bincount(rows, minlength=flat.shape[0])
        self.off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        self.bin = bins.astype(np.int32)
        self.cnt = flat[rows, bins].astype(np.float64)
        g = np.ones((self.hh, self.ww)) if gain is None else np.asarray(gain, np.float64)
        self.gain = np.ascontiguousarray(g.reshape(self.hh, self.ww))
        self.irf_idx = None if irf_idx is None else np.ascontiguousarray(
            np.asarray(irf_idx, np.uint8).reshape(self.hh, self.ww))

    def c(self):
        return Frame(self.hh, self.ww, self.tt, _ptr(self.off, C.c_int64),
                     _ptr(self.bin, C.c_int32), _ptr(self.cnt, C.c_double),
                     _ptr(self.gain, C.c_double),
                     None if self.irf_idx is None else _ptr(self.irf_idx, C.c_uint8))


# ---------------------------------------------------------------------------
# functions
# ---------------------------------------------------------------------------

def philox(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def poisson_fixed(u, p0, mu):
    return int(lib().or_poisson_fixed(C.c_uint32(int(u)), C.c_uint64(int(p0)), C.c_uint64(int(mu))))


def synthesize(tab: dict, seed=None) -> np.ndarray:
    """Histogram [H][W][T] uint16 from the integer tables of scenes.sampling_tables."""
    h, w, t = tab["h"], tab["w"], tab["t"]
    out = np.zeros((h, w, t), np.uint16)
    seed = tab["seed"] if seed is None else seed
    lib().or_synthesize(h, w, t, tab["n_comp"],
                        _ptr(tab["depth_int"], C.c_int32), _ptr(tab["depth_split"], C.c_uint32),
                        _ptr(tab["n_parts"], C.c_uint32), _ptr(tab["p0"], C.c_uint64),
                        _ptr(tab["mu"], C.c_uint64), _ptr(tab["irf_cdf"], C.c_uint32),
                        tab["irf_len"], tab["irf_origin"], C.c_uint64(int(seed)),
                        _ptr(out, C.c_uint16))
    return out


def irf_eval(irf: OIrf, x):
    h = C.c_double()
    dh = C.c_double()
    lib().or_irf_eval(C.byref(irf.c()), C.c_double(float(x)), C.byref(h), C.byref(dh))
    return h.value, dh.value


def nll_dense(z, gain, st: OState, irf, lam_floor, irf_idx=None, up=1):
    z = np.ascontiguousarray(z, np.float64)
    h, w, t = z.shape
    g = np.ascontiguousarray(np.ones((h, w)) if gain is None else gain, np.float64)
    idx = None if irf_idx is None else np.ascontiguousarray(np.asarray(irf_idx, np.uint8).reshape(h, w))
    return lib().or_nll_dense_idx(h, w, t, _ptr(z, C.c_double), _ptr(g, C.c_double),
                                  None if idx is None else _ptr(idx, C.c_uint8), int(up),
                                  C.byref(st.c()), _irfs(irf), C.c_double(lam_floor))


def gradients(fr: OFrame, st: OState, irf, prm: dict):
    gt = np.zeros(st.t.shape)
    gr = np.zeros(st.t.shape)
    gb = np.zeros((fr.hh, fr.ww))
    p = make_params(prm)
    lib().or_gradients(C.byref(fr.c()), C.byref(st.c()), _irfs(irf), C.byref(p),
                       _ptr(gt, C.c_double), _ptr(gr, C.c_double), _ptr(gb, C.c_double))
    return gt, gr, gb


def lmf_kernel(irf: OIrf, delta_rel, frac_bits):
    k = np.zeros(len(irf.h), np.int32)
    lib().or_lmf_kernel(C.byref(irf.c()), C.c_double(_f32(delta_rel)), int(frac_bits),
                        _ptr(k, C.c_int32))
    return k


def lmf(z_row, kern, origin):
    z = np.ascontiguousarray(z_row, np.uint16)
    kern = np.ascontiguousarray(kern, np.int32)
    t = z.shape[0]
    y = np.zeros(t, np.int64)
    wc = np.zeros(t, np.int64)
    lib().or_lmf(_ptr(z, C.c_uint16), t, _ptr(kern, C.c_int32), len(kern), int(origin),
                 _ptr(y, C.c_int64), _ptr(wc, C.c_int64))
    return y, wc


def peaks(y, wc, sep, min_photons, kmax):
    y = np.ascontiguousarray(y, np.int64)
    wc = np.ascontiguousarray(wc, np.int64)
    taus = np.zeros(16, np.int32)
    n = lib().or_peaks(_ptr(y, C.c_int64), _ptr(wc, C.c_int64), len(y), int(sep),
                       int(min_photons), int(kmax), _ptr(taus, C.c_int32))
    return taus[:n].copy()


def init(dense, gain, irf, prm: dict, irf_idx=None) -> OState:
    """Initialisation; irf is an OIrf or a list of them with irf_idx [h][w]
    selecting each pixel's."""
    dense = np.ascontiguousarray(dense, np.uint16)
    h, w, t = dense.shape
    g = np.ascontiguousarray(np.ones((h, w)) if gain is None else gain, np.float64)
    idx = None if irf_idx is None else np.ascontiguousarray(np.asarray(irf_idx, np.uint8).reshape(h, w))
    st = new_state(prm["k_max"], h, w, int(prm.get("upsample", 1)))
    p = make_params(prm)
    lib().or_init_idx(_ptr(dense, C.c_uint16), _ptr(g, C.c_double),
                      None if idx is None else _ptr(idx, C.c_uint8), h, w, t, _irfs(irf),
                      C.byref(p), C.byref(st.c()))
    return st


def t_step(fr, irf, prm, st):
    lib().or_t_step(C.byref(fr.c()), _irfs(irf), C.byref(make_params(prm)), C.byref(st.c()))


def r_step(fr, irf, prm, st):
    lib().or_r_step(C.byref(fr.c()), _irfs(irf), C.byref(make_params(prm)), C.byref(st.c()))


def b_step(fr, irf, prm, st):
    lib().or_b_step(C.byref(fr.c()), _irfs(irf), C.byref(make_params(prm)), C.byref(st.c()))


def apss(h, w, t, prm, st):
    lib().or_apss(h, w, t, C.byref(make_params(prm)), C.byref(st.c()))


def plane(h, w, t, prm, st):
    lib().or_plane(h, w, t, C.byref(make_params(prm)), C.byref(st.c()))


def bilateral(h, w, t, prm, st):
    lib().or_bilateral(h, w, t, C.byref(make_params(prm)), C.byref(st.c()))


def int_lowpass(h, w, prm, st):
    lib().or_int_lowpass(h, w, C.byref(make_params(prm)), C.byref(st.c()))


def bkg_lowpass(h, w, prm, b):
    lib().or_bkg_lowpass(h, w, C.byref(make_params(prm)), _ptr(b, C.c_double))


def depth_denoise(h, w, t, prm, st):
    """The depth block's denoiser selected by prm["depth_denoiser"]."""
    lib().or_depth_denoise(int(h), int(w), int(t), C.byref(make_params(prm)), C.byref(st.c()))


def palm(fr, irf, prm, st, n_iter):
    lib().or_palm(C.byref(fr.c()), _irfs(irf), C.byref(make_params(prm)),
                  C.byref(st.c()), int(n_iter))


def reconstruct(dense, irf, prm: dict, gain=None, irf_idx=None) -> OState:
    """The whole method; irf is an OIrf or a list of them with irf_idx [h][w]
    selecting each pixel's."""
    dense = np.ascontiguousarray(dense, np.uint16)
    h, w, t = dense.shape
    fr = OFrame(dense, gain, irf_idx)
    st = new_state(prm["k_max"], h, w, int(prm.get("upsample", 1)))
    lib().or_reconstruct(_ptr(dense, C.c_uint16), C.byref(fr.c()), _irfs(irf),
                         C.byref(make_params(prm)), C.byref(st.c()))
    return st


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops in this process."""
    lib().or_set_num_threads(int(n))


# ---------------------------------------------------------------------------
# learned depth denoiser (extension; net.c)

NET_LAYERS = 4


def net_nparams() -> int:
    return int(lib().or_net_nparams())


def net_offset(layer: int, bias: bool) -> int:
    return int(lib().or_net_offset(int(layer), int(bool(bias))))


def net_channels():
    return [(int(lib().or_net_cin(l)), int(lib().or_net_cout(l))) for l in range(NET_LAYERS)]


def bf16(x):
    a = np.array(x, dtype=np.float64, copy=True)
    lib().or_bf16_round(_ptr(a, C.c_double), C.c_long(a.size))
    return a


def net_features(st: OState, scale: float) -> np.ndarray:
    k, h, w = st.t.shape
    x = np.zeros((6, h, w), np.float64)
    lib().or_net_features(int(h), int(w), C.byref(st.c()), C.c_double(scale), _ptr(x, C.c_double))
    return x


def _acts_size(n, h, w):
    return sum(n * ci * h * w for ci, _ in net_channels())


def net_forward(theta, x, bf16_round=True):
    """x [n][6][h][w] -> (acts, y [n][2][h][w])."""
    theta = np.ascontiguousarray(theta, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    n, c, h, w = x.shape
    acts = np.zeros(_acts_size(n, h, w), np.float64)
    y = np.zeros((n, 2, h, w), np.float64)
    lib().or_net_forward(int(n), int(h), int(w), _ptr(theta, C.c_double), _ptr(x, C.c_double),
                         int(bool(bf16_round)), _ptr(acts, C.c_double), _ptr(y, C.c_double))
    return acts, y


def net_loss(y, target, mask):
    y = np.ascontiguousarray(y, np.float64)
    target = np.ascontiguousarray(target, np.float64)
    mask = np.ascontiguousarray(mask, np.uint8)
    n, _, h, w = y.shape
    dy = np.zeros_like(y)
    loss = lib().or_net_loss(int(n), int(h), int(w), _ptr(y, C.c_double), _ptr(target, C.c_double),
                             _ptr(mask, C.c_uint8), _ptr(dy, C.c_double))
    return float(loss), dy


def net_backward(theta, acts, dy, bf16_round=True, want_dx=False):
    theta = np.ascontiguousarray(theta, np.float64)
    dy = np.ascontiguousarray(dy, np.float64)
    n, _, h, w = dy.shape
    dtheta = np.zeros_like(theta)
    dx = np.zeros((n, 6, h, w), np.float64) if want_dx else None
    lib().or_net_backward(int(n), int(h), int(w), _ptr(theta, C.c_double), _ptr(acts, C.c_double),
                          _ptr(dy, C.c_double), int(bool(bf16_round)), _ptr(dtheta, C.c_double),
                          _ptr(dx, C.c_double) if want_dx else None)
    return dtheta, dx


def adamw(theta, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step, in place on theta, m, v (float64 arrays)."""
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, np.float64)
    lib().or_adamw(_ptr(theta, C.c_double), _ptr(g, C.c_double), _ptr(m, C.c_double), _ptr(v, C.c_double),
                   int(step), C.c_double(lr), C.c_double(beta1), C.c_double(beta2), C.c_double(eps),
                   C.c_double(wd))


def learned_depth(h, w, t, prm: dict, st: OState):
    lib().or_learned_depth(int(h), int(w), int(t), C.byref(make_params(prm)), C.byref(st.c()))
