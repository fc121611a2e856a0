"""Thin Python binding of the rt3d C ABI (include/rt3d.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides device memory and streams.  The functions
named rt3d_* mirror the C entry points one to one; `Context` bundles them
with torch-tensor allocation for convenience.  There is no CPU fallback: if
the compiled library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "librt3d.so")

RT3D_OK = 0
RT3D_E_INVALID = -1
RT3D_E_NOMEM = -2
RT3D_E_CUDA = -3
RT3D_E_TIMEOUT = -4
RT3D_E_UNIMPL = -5
RT3D_E_CAPACITY = -6
RT3D_E_RANGE = -7

MAX_K = 4
MAX_BATCH = 64


class Rt3dError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: rt3d status {status} ({status_str(status)})")


class Config(C.Structure):
    _fields_ = [("max_h", C.c_int32), ("max_w", C.c_int32), ("max_t", C.c_int32),
                ("k_max", C.c_int32), ("max_batch", C.c_int32), ("max_entries", C.c_int64),
                ("device", C.c_int32), ("mem_budget", C.c_int64)]


class Irf(C.Structure):
    _fields_ = [("samples", C.POINTER(C.c_double)), ("len", C.c_int32), ("origin", C.c_int32)]


class Frame(C.Structure):
    _fields_ = [("h", C.c_int32), ("w", C.c_int32), ("t", C.c_int32),
                ("dense", C.c_void_p), ("csr_off", C.c_void_p), ("csr_ent", C.c_void_p),
                ("gain", C.c_void_p), ("irf_index", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("n_iter", C.c_int32), ("k_max", C.c_int32),
                ("t_step", C.c_float), ("r_step", C.c_float), ("b_step", C.c_float),
                ("dt_max", C.c_float), ("eps_r", C.c_float), ("eps_b", C.c_float),
                ("b_floor", C.c_float), ("lam_floor", C.c_float),
                ("pixel_pitch", C.c_float), ("apss_radius", C.c_float),
                ("win_r", C.c_int32), ("apss_min_nb", C.c_int32),
                ("int_radius", C.c_float), ("r_min", C.c_float), ("merge_dist", C.c_float),
                ("depth_denoiser", C.c_int32), ("intensity_denoiser", C.c_int32),
                ("bkg_mode", C.c_int32), ("bkg_sigma", C.c_float), ("bkg_radius", C.c_int32),
                ("lmf_delta_rel", C.c_float), ("lmf_frac_bits", C.c_int32),
                ("peak_min_photons", C.c_int32), ("peak_sep", C.c_int32),
                ("lmf_precision", C.c_int32), ("warm_start", C.c_int32),
                ("net_scale", C.c_float), ("net_fallback", C.c_float), ("apss_fp64", C.c_int32),
                ("upsample", C.c_int32)]


class AdamW(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("weight_decay", C.c_float)]


NET_PARAMS = 45074


class Result(C.Structure):
    _fields_ = [("t", C.c_void_p), ("r", C.c_void_p), ("alive", C.c_void_p), ("b", C.c_void_p),
                ("n_points", C.c_void_p)]


class Scene(C.Structure):
    _fields_ = [("h", C.c_int32), ("w", C.c_int32), ("t", C.c_int32), ("n_comp", C.c_int32),
                ("depth_int", C.c_void_p), ("depth_split", C.c_void_p), ("n_parts", C.c_void_p),
                ("p0", C.c_void_p), ("mu", C.c_void_p), ("irf_cdf", C.c_void_p),
                ("irf_len", C.c_int32), ("irf_origin", C.c_int32)]


_lib = None
_P = C.c_void_p


def lib():
    """Load lib/librt3d.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"rt3d CUDA library not built: {LIB_PATH} is missing "
                           "(run __graft_entry__.build() or python paper_1905_06700_b300/build.py)")
    L = C.CDLL(LIB_PATH)
    sig = {
        "rt3d_status_str": (C.c_char_p, [C.c_int]),
        "rt3d_version": (C.c_int, []),
        "rt3d_default_params": (C.c_int, [C.POINTER(Params)]),
        "rt3d_validate": (C.c_int, [C.POINTER(Config), C.POINTER(Frame), C.POINTER(Params)]),
        "rt3d_create": (C.c_int, [C.POINTER(Config), C.POINTER(Irf), C.POINTER(_P)]),
        "rt3d_workspace_bytes": (C.c_int, [C.POINTER(Config), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "rt3d_net_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(_P)]),
        "rt3d_net_destroy": (None, [_P]),
        "rt3d_net_set_params": (C.c_int, [_P, _P]),
        "rt3d_net_get_params": (C.c_int, [_P, _P]),
        "rt3d_net_features": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P, C.c_float, _P, _P]),
        "rt3d_net_forward": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P]),
        "rt3d_net_gradient": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, _P, _P]),
        "rt3d_net_train_step": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P, C.POINTER(AdamW), _P, _P]),
        "rt3d_set_depth_net": (C.c_int, [_P, _P]),
        "rt3d_destroy": (None, [_P]),
        "rt3d_synthesize": (C.c_int, [_P, C.POINTER(Scene), C.c_uint64, _P, _P]),
        "rt3d_compact": (C.c_int, [_P, C.POINTER(Frame), _P, _P, C.c_int64,
                                   C.POINTER(C.c_int64), _P]),
        "rt3d_lmf": (C.c_int, [_P, C.POINTER(Frame), C.POINTER(Params), _P, _P]),
        "rt3d_init": (C.c_int, [_P, C.POINTER(Frame), C.POINTER(Params), C.POINTER(Result), _P]),
        "rt3d_reconstruct": (C.c_int, [_P, C.POINTER(Frame), C.POINTER(Params),
                                       C.POINTER(Result), _P]),
        "rt3d_reconstruct_batch": (C.c_int, [_P, C.c_int, C.POINTER(Frame), C.POINTER(Params),
                                             C.POINTER(Result), _P]),
        "rt3d_reconstruct_batch_host": (C.c_int, [_P, C.c_int, C.POINTER(Frame), C.POINTER(Params),
                                                   C.POINTER(Result), _P]),
        "rt3d_reconstruct_host": (C.c_int, [_P, C.POINTER(Frame), C.POINTER(Params),
                                            C.POINTER(Result), _P]),
        "rt3d_phase": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(Frame), C.POINTER(Params),
                                 C.POINTER(Result), _P]),
        "rt3d_device_status": (C.c_int, [_P, _P]),
        "rt3d_launch_count": (C.c_int64, [_P]),
        "rt3d_set_wait_limit": (C.c_int, [_P, C.c_int64]),
        "rt3d_set_irfs": (C.c_int, [_P, C.c_int, C.POINTER(Irf)]),
        "rt3d_set_profiling": (C.c_int, [_P, C.c_int]),
        "rt3d_kernel_times": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                        C.c_int, C.c_int]),
        "rt3d_get_sparse": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64,
                                      C.POINTER(C.c_int64), _P]),
        "rt3d_reconstruct_noalloc": (C.c_int, [C.POINTER(Irf), C.POINTER(Frame),
                                               C.POINTER(Params), C.POINTER(Result), _P]),
        "rt3d_noalloc_status": (C.c_int, [_P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def status_str(status: int) -> str:
    try:
        return lib().rt3d_status_str(status).decode()
    except Exception:  # library missing: still format the error
        return "unknown"


def check(status: int, what: str):
    if status != RT3D_OK:
        raise Rt3dError(status, what)


# ---- one-to-one wrappers of the C entry points --------------------------------

def rt3d_version() -> int:
    return lib().rt3d_version()


def rt3d_default_params() -> Params:
    p = Params()
    check(lib().rt3d_default_params(C.byref(p)), "rt3d_default_params")
    return p


def rt3d_validate(cfg: Config, frame: Optional[Frame], params: Optional[Params]) -> int:
    return lib().rt3d_validate(C.byref(cfg), C.byref(frame) if frame else None,
                               C.byref(params) if params else None)


def rt3d_create(cfg: Config, irf_samples, irf_origin: int):
    samples = np.ascontiguousarray(irf_samples, dtype=np.float64)
    irf = Irf(samples.ctypes.data_as(C.POINTER(C.c_double)), len(samples), int(irf_origin))
    h = _P()
    check(lib().rt3d_create(C.byref(cfg), C.byref(irf), C.byref(h)), "rt3d_create")
    return h


def rt3d_destroy(h):
    lib().rt3d_destroy(h)


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def workspace_bytes(cfg: Config):
    """(bytes, entry capacity) of the workspace rt3d_create(cfg) would take."""
    b = C.c_int64()
    e = C.c_int64()
    check(lib().rt3d_workspace_bytes(C.byref(cfg), C.byref(b), C.byref(e)), "rt3d_workspace_bytes")
    return int(b.value), int(e.value)


def params_from(d) -> Params:
    """Params from a dict (missing keys take the library defaults)."""
    if isinstance(d, Params):
        return d
    p = rt3d_default_params()
    for name, ctype in Params._fields_:
        if name in d:
            setattr(p, name, int(d[name]) if ctype is C.c_int32 else float(d[name]))
    return p


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Context:
    """A library context plus torch-tensor marshalling for its entry points."""

    def __init__(self, max_h: int, max_w: int, max_t: int, k_max: int, irf_samples, irf_origin: int,
                 max_batch: int = 1, max_entries: int = 0, device: int = 0, mem_budget: int = 0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.cfg = Config(max_h, max_w, max_t, k_max, max_batch, max_entries, device, mem_budget)
        self.k_max = k_max
        self.handle = rt3d_create(self.cfg, irf_samples, irf_origin)

    def close(self):
        if getattr(self, "handle", None):
            rt3d_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- frames / results -------------------------------------------------------
    def frame(self, dense=None, csr=None, gain=None, shape=None, irf_index=None) -> Frame:
        if dense is not None:
            h, w, t = dense.shape
        else:
            h, w, t = shape
        off, ent = (csr if csr is not None else (None, None))
        return Frame(h, w, t, _ptr(dense), _ptr(off), _ptr(ent), _ptr(gain), _ptr(irf_index))

    def set_irfs(self, irfs):
        """rt3d_set_irfs: irfs = [(samples, origin), ...], response i for
        pixels whose irf_index is i."""
        arr = (Irf * len(irfs))()
        keep = []
        for i, (samples, origin) in enumerate(irfs):
            a = np.ascontiguousarray(samples, np.float64)
            keep.append(a)
            arr[i] = Irf(a.ctypes.data_as(C.POINTER(C.c_double)), len(a), int(origin))
        check(lib().rt3d_set_irfs(self.handle, len(irfs), arr), "rt3d_set_irfs")

    def new_result(self, h, w, k=None, up=1):
        """Result tensors of an h x w frame: points on the world grid (up times
        finer with super-resolution), background per pixel."""
        torch = self.torch
        k = k or self.k_max
        d = self.device
        return dict(t=torch.zeros((k, h * up, w * up), dtype=torch.float32, device=d),
                    r=torch.zeros((k, h * up, w * up), dtype=torch.float32, device=d),
                    alive=torch.zeros((k, h * up, w * up), dtype=torch.uint8, device=d),
                    b=torch.zeros((h, w), dtype=torch.float32, device=d),
                    n_points=torch.zeros(1, dtype=torch.int32, device=d))

    @staticmethod
    def result_struct(res: dict) -> Result:
        return Result(_ptr(res["t"]), _ptr(res["r"]), _ptr(res["alive"]), _ptr(res["b"]),
                      _ptr(res.get("n_points")))

    # -- entry points -------------------------------------------------------------
    def synthesize(self, tables: dict, seed: Optional[int] = None, out=None, stream=None):
        torch = self.torch
        d = self.device
        h, w, t = tables["h"], tables["w"], tables["t"]

        def up(a, dt):
            return torch.from_numpy(np.ascontiguousarray(a).view(dt)).to(d)
        keep = dict(depth_int=up(tables["depth_int"], np.int32),
                    depth_split=up(tables["depth_split"], np.int32),
                    n_parts=up(tables["n_parts"], np.int32),
                    p0=up(tables["p0"], np.int64), mu=up(tables["mu"], np.int64),
                    irf_cdf=up(tables["irf_cdf"] if len(tables["irf_cdf"]) else np.zeros(1, np.uint32),
                               np.int32))
        sc = Scene(h, w, t, tables["n_comp"], _ptr(keep["depth_int"]), _ptr(keep["depth_split"]),
                   _ptr(keep["n_parts"]), _ptr(keep["p0"]), _ptr(keep["mu"]), _ptr(keep["irf_cdf"]),
                   tables["irf_len"], tables["irf_origin"])
        if out is None:
            out = torch.empty((h, w, t), dtype=torch.uint16, device=d)
        seed = tables["seed"] if seed is None else seed
        check(lib().rt3d_synthesize(self.handle, C.byref(sc), C.c_uint64(int(seed)), _ptr(out),
                                    _stream(stream)), "rt3d_synthesize")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return out

    def compact(self, dense, capacity=None, stream=None):
        torch = self.torch
        h, w, t = dense.shape
        if capacity is None:
            capacity = h * w * t
        off = torch.empty(h * w + 1, dtype=torch.int32, device=self.device)
        ent = torch.empty(max(int(capacity), 1), dtype=torch.int32, device=self.device)
        nnz = C.c_int64()
        fr = self.frame(dense)
        check(lib().rt3d_compact(self.handle, C.byref(fr), _ptr(off), _ptr(ent), int(capacity),
                                 C.byref(nnz), _stream(stream)), "rt3d_compact")
        return off, ent[: nnz.value]

    def lmf(self, params, dense=None, csr=None, shape=None, stream=None):
        torch = self.torch
        fr = self.frame(dense, csr, shape=shape)
        y = torch.empty((fr.h, fr.w, fr.t), dtype=torch.int32, device=self.device)
        p = params_from(params)
        check(lib().rt3d_lmf(self.handle, C.byref(fr), C.byref(p), _ptr(y), _stream(stream)), "rt3d_lmf")
        return y

    def init(self, params, dense=None, csr=None, gain=None, shape=None, out=None, stream=None,
             irf_index=None):
        fr = self.frame(dense, csr, gain, shape, irf_index)
        p = params_from(params)
        out = out or self.new_result(fr.h, fr.w, p.k_max, p.upsample)
        rs = self.result_struct(out)
        check(lib().rt3d_init(self.handle, C.byref(fr), C.byref(p), C.byref(rs), _stream(stream)),
              "rt3d_init")
        return out

    def reconstruct(self, params, dense=None, csr=None, gain=None, shape=None, out=None, stream=None,
             irf_index=None):
        fr = self.frame(dense, csr, gain, shape, irf_index)
        p = params_from(params)
        out = out or self.new_result(fr.h, fr.w, p.k_max, p.upsample)
        rs = self.result_struct(out)
        check(lib().rt3d_reconstruct(self.handle, C.byref(fr), C.byref(p), C.byref(rs),
                                     _stream(stream)), "rt3d_reconstruct")
        return out

    def reconstruct_batch(self, params, frames: Sequence[dict], outs=None, stream=None):
        p = params_from(params)
        n = len(frames)
        fa = (Frame * n)()
        for i, f in enumerate(frames):
            fa[i] = self.frame(f.get("dense"), f.get("csr"), f.get("gain"), f.get("shape"), f.get("irf_index"))
        if outs is None:
            outs = [self.new_result(fa[i].h, fa[i].w, p.k_max, p.upsample) for i in range(n)]
        ra = (Result * n)(*[self.result_struct(o) for o in outs])
        check(lib().rt3d_reconstruct_batch(self.handle, n, fa, C.byref(p), ra, _stream(stream)),
              "rt3d_reconstruct_batch")
        return outs

    def phase(self, phase: int, first: int, params, csr, state: dict, gain=None, shape=None, stream=None,
              irf_index=None):
        fr = self.frame(None, csr, gain, shape, irf_index)
        p = params_from(params)
        rs = self.result_struct(state)
        check(lib().rt3d_phase(self.handle, int(phase), int(first), C.byref(fr), C.byref(p),
                               C.byref(rs), _stream(stream)), "rt3d_phase")
        return state

    def set_depth_net(self, net):
        """Attach a Net as the loop's learned depth denoiser (None detaches)."""
        check(lib().rt3d_set_depth_net(self.handle, net.handle if net is not None else None),
              "rt3d_set_depth_net")
        self._net = net

    def device_status(self, stream=None) -> int:
        return lib().rt3d_device_status(self.handle, _stream(stream))

    def launch_count(self) -> int:
        return int(lib().rt3d_launch_count(self.handle))

    def set_wait_limit(self, ns: int):
        """Bound of the tensor-core kernels' device-side waits (rt3d_set_wait_limit)."""
        check(lib().rt3d_set_wait_limit(self.handle, int(ns)), "rt3d_set_wait_limit")

    def set_profiling(self, on: bool):
        check(lib().rt3d_set_profiling(self.handle, int(on)), "rt3d_set_profiling")

    def kernel_times(self, reset=False):
        ms = (C.c_double * 9)()
        n = (C.c_int64 * 9)()
        check(lib().rt3d_kernel_times(self.handle, ms, n, 9, int(reset)), "rt3d_kernel_times")
        names = ["init", "phase_a", "phase_b", "phase_c", "final", "synth", "compact", "net", "init_tc"]
        return {names[i]: (ms[i], n[i]) for i in range(9)}

    def get_sparse(self, n_pix: int, n_ent: int, stream=None):
        seg = np.zeros((n_pix, 2), np.uint32)
        ent = np.zeros(max(n_ent, 1), np.uint32)
        used = C.c_int64()
        check(lib().rt3d_get_sparse(self.handle, seg.ctypes.data_as(C.c_void_p), n_pix,
                                    ent.ctypes.data_as(C.c_void_p), n_ent, C.byref(used),
                                    _stream(stream)), "rt3d_get_sparse")
        return seg, ent[:n_ent], used.value


def _host_ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def reconstruct_host(ctx: Context, params, dense: np.ndarray, gain: Optional[np.ndarray] = None,
                     csr: Optional[tuple] = None, out: Optional[dict] = None, stream=None,
                     irf_index: Optional[np.ndarray] = None) -> dict:
    """rt3d_reconstruct_host: HOST numpy buffers in and out (copies inside the call)."""
    p = params_from(params)
    h, w, t = dense.shape if dense is not None else csr[2]
    dense = None if dense is None else np.ascontiguousarray(dense, np.uint16)
    gain = None if gain is None else np.ascontiguousarray(gain, np.float32)
    irf_index = None if irf_index is None else np.ascontiguousarray(irf_index, np.uint8)
    off = ent = None
    if csr is not None:
        off = np.ascontiguousarray(csr[0], np.uint32)
        ent = np.ascontiguousarray(csr[1], np.uint32)
    fr = Frame(h, w, t, _host_ptr(dense), _host_ptr(off), _host_ptr(ent), _host_ptr(gain), _host_ptr(irf_index))
    k = p.k_max
    if out is None:
        out = dict(t=np.zeros((k, h, w), np.float32), r=np.zeros((k, h, w), np.float32),
                   alive=np.zeros((k, h, w), np.uint8), b=np.zeros((h, w), np.float32),
                   n_points=np.zeros(1, np.int32))
    rs = Result(_host_ptr(out["t"]), _host_ptr(out["r"]), _host_ptr(out["alive"]),
                _host_ptr(out["b"]), _host_ptr(out.get("n_points")))
    check(lib().rt3d_reconstruct_host(ctx.handle, C.byref(fr), C.byref(p), C.byref(rs),
                                      _stream(stream)), "rt3d_reconstruct_host")
    return out


def reconstruct_batch_host(ctx: Context, params, frames: Sequence[dict], outs: Optional[Sequence[dict]] = None,
                           stream=None) -> list:
    """rt3d_reconstruct_batch_host: n frames of HOST numpy buffers in, HOST
    results out, one batched reconstruction.  Each frame dict holds `dense`
    ([h][w][t] uint16) and/or `csr` ((offsets, entries, (h, w, t))), and
    optionally `gain` and `irf_index`; page-locked arrays give full link
    bandwidth."""
    p = params_from(params)
    k = p.k_max
    keep, frs, rss = [], [], []
    outs = list(outs) if outs is not None else [None] * len(frames)
    for i, f in enumerate(frames):
        dense = f.get("dense")
        csr = f.get("csr")
        h, w, t = dense.shape if dense is not None else csr[2]
        dense = None if dense is None else np.ascontiguousarray(dense, np.uint16)
        gain = None if f.get("gain") is None else np.ascontiguousarray(f["gain"], np.float32)
        idx = None if f.get("irf_index") is None else np.ascontiguousarray(f["irf_index"], np.uint8)
        off = ent = None
        if csr is not None:
            off = np.ascontiguousarray(csr[0], np.uint32)
            ent = np.ascontiguousarray(csr[1], np.uint32)
        keep += [dense, gain, off, ent, idx]
        frs.append(Frame(h, w, t, _host_ptr(dense), _host_ptr(off), _host_ptr(ent), _host_ptr(gain),
                         _host_ptr(idx)))
        if outs[i] is None:
            outs[i] = dict(t=np.zeros((k, h, w), np.float32), r=np.zeros((k, h, w), np.float32),
                           alive=np.zeros((k, h, w), np.uint8), b=np.zeros((h, w), np.float32),
                           n_points=np.zeros(1, np.int32))
        o = outs[i]
        rss.append(Result(_host_ptr(o["t"]), _host_ptr(o["r"]), _host_ptr(o["alive"]), _host_ptr(o["b"]),
                          _host_ptr(o.get("n_points"))))
    fa = (Frame * len(frs))(*frs)
    ra = (Result * len(rss))(*rss)
    check(lib().rt3d_reconstruct_batch_host(ctx.handle, len(frs), fa, C.byref(p), ra, _stream(stream)),
          "rt3d_reconstruct_batch_host")
    return outs


def rt3d_reconstruct_noalloc(irf_samples, irf_origin: int, frame: Frame, params, result: Result,
                             stream=None) -> int:
    """The whole method with the library's static scratch: no context and no
    allocation (for callers that must not allocate device memory while they
    run).  Returns the rt3d status."""
    samples = np.ascontiguousarray(irf_samples, dtype=np.float64)
    irf = Irf(samples.ctypes.data_as(C.POINTER(C.c_double)), len(samples), int(irf_origin))
    p = params_from(params)
    return lib().rt3d_reconstruct_noalloc(C.byref(irf), C.byref(frame), C.byref(p),
                                          C.byref(result), _stream(stream))


def rt3d_noalloc_status(stream=None) -> int:
    """Device status of the last allocation-free call on the current device
    (synchronises; clears the word)."""
    return lib().rt3d_noalloc_status(_stream(stream))


class Net:
    """The learned depth denoiser's network (device parameters, AdamW state and
    a training workspace for up to max_images images of max_h x max_w)."""

    def __init__(self, max_images: int, max_h: int, max_w: int, device: int = 0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        h = _P()
        check(lib().rt3d_net_create(int(device), int(max_images), int(max_h), int(max_w), C.byref(h)),
              "rt3d_net_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().rt3d_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        a = np.ascontiguousarray(np.asarray(theta, np.float32))
        assert a.size == NET_PARAMS
        check(lib().rt3d_net_set_params(self.handle, a.ctypes.data_as(_P)), "rt3d_net_set_params")

    def get_params(self) -> np.ndarray:
        a = np.zeros(NET_PARAMS, np.float32)
        check(lib().rt3d_net_get_params(self.handle, a.ctypes.data_as(_P)), "rt3d_net_get_params")
        return a

    def features(self, t, r, alive, scale: float, stream=None):
        """t, r, alive [n][k][h][w] (device) -> x [n][6][h][w]."""
        n, k, h, w = t.shape
        x = self.torch.empty((n, 6, h, w), dtype=self.torch.float32, device=self.device)
        check(lib().rt3d_net_features(self.handle, n, k, h, w, _ptr(t), _ptr(r), _ptr(alive), float(scale),
                                      _ptr(x), _stream(stream)), "rt3d_net_features")
        return x

    def forward(self, x, stream=None):
        n, _, h, w = x.shape
        y = self.torch.empty((n, 2, h, w), dtype=self.torch.float32, device=self.device)
        check(lib().rt3d_net_forward(self.handle, n, h, w, _ptr(x), _ptr(y), _stream(stream)),
              "rt3d_net_forward")
        return y

    def gradient(self, x, target, mask, stream=None):
        n, _, h, w = x.shape
        g = self.torch.empty(NET_PARAMS, dtype=self.torch.float32, device=self.device)
        loss = self.torch.empty(1, dtype=self.torch.float32, device=self.device)
        check(lib().rt3d_net_gradient(self.handle, n, h, w, _ptr(x), _ptr(target), _ptr(mask), _ptr(g),
                                      _ptr(loss), _stream(stream)), "rt3d_net_gradient")
        return g, loss

    def train_step(self, x, target, mask, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0,
                   loss=None, stream=None):
        n, _, h, w = x.shape
        opt = AdamW(lr, beta1, beta2, eps, weight_decay)
        check(lib().rt3d_net_train_step(self.handle, n, h, w, _ptr(x), _ptr(target), _ptr(mask), C.byref(opt),
                                        _ptr(loss), _stream(stream)), "rt3d_net_train_step")
