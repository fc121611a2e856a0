"""The C-ABI library loads, exports every declared entry point, and its host-only
logic (validation, defaults, status strings) behaves; no GPU needed."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_1905_06700_b300 import build as B
from paper_1905_06700_b300 import rt3d as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rt3d.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    return R.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rt3d_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", R.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(rt3d_\w+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(L, n)


STRUCTS = {
    "rt3d_config": R.Config, "rt3d_irf": R.Irf, "rt3d_frame": R.Frame,
    "rt3d_params": R.Params, "rt3d_result": R.Result, "rt3d_scene": R.Scene,
}


def test_binding_struct_layouts_match_the_header():
    """sizeof/offsetof of every ABI struct, as gcc sees the header, equal the
    ctypes mirrors used by the binding."""
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', 'int main(void){']
    for cname, py in STRUCTS.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-o", exe, src], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    for line in out.strip().splitlines():
        cname, field, val = line.split()
        py = STRUCTS[cname]
        want = C.sizeof(py) if field == "size" else getattr(py, field).offset
        assert int(val) == want, (cname, field, val, want)


def test_status_strings_and_defaults(L):
    assert R.rt3d_version() == 1
    assert R.status_str(0) == "ok"
    assert "capacity" in R.status_str(R.RT3D_E_CAPACITY)
    p = R.rt3d_default_params()
    assert p.n_iter == 20 and p.win_r == 3 and p.depth_denoiser == 1


def _cfg(**kw):
    d = dict(max_h=64, max_w=64, max_t=1024, k_max=3, max_batch=4, max_entries=0, device=0)
    d.update(kw)
    return R.Config(**d)


def _frame(**kw):
    d = dict(h=32, w=32, t=1024, dense=C.c_void_p(0x1000), csr_off=None, csr_ent=None, gain=None)
    d.update(kw)
    return R.Frame(**d)


def test_validation_accepts_a_good_call(L):
    p = R.rt3d_default_params()
    assert R.rt3d_validate(_cfg(), _frame(), p) == R.RT3D_OK


@pytest.mark.parametrize("cfg_kw", [dict(max_h=0), dict(k_max=5), dict(max_batch=65),
                                    dict(max_t=70000), dict(max_entries=-1), dict(device=-1)])
def test_validation_rejects_bad_configs(L, cfg_kw):
    assert R.rt3d_validate(_cfg(**cfg_kw), None, None) == R.RT3D_E_INVALID


@pytest.mark.parametrize("fr_kw", [dict(h=0), dict(w=65), dict(t=1025), dict(dense=None),
                                   dict(dense=None, csr_off=C.c_void_p(0x10)),
                                   dict(csr_ent=C.c_void_p(0x10))])
def test_validation_rejects_bad_frames(L, fr_kw):
    assert R.rt3d_validate(_cfg(), _frame(**fr_kw), R.rt3d_default_params()) == R.RT3D_E_INVALID


@pytest.mark.parametrize("field,value", [("n_iter", -1), ("k_max", 0), ("k_max", 4), ("t_step", 0.0),
                                         ("r_min", 0.0), ("win_r", 5), ("bkg_radius", 16),
                                         ("lmf_frac_bits", 13), ("peak_min_photons", 256),
                                         ("depth_denoiser", 5), ("apss_fp64", 2), ("apss_radius", float("nan")),
                                         ("lmf_delta_rel", 0.0)])
def test_validation_rejects_bad_params(L, field, value):
    p = R.rt3d_default_params()
    setattr(p, field, value)
    assert R.rt3d_validate(_cfg(), _frame(), p) == R.RT3D_E_INVALID


def test_create_without_usable_device_fails_cleanly(L):
    """With no GPU (or a bad ordinal) creation returns an error, never crashes."""
    import numpy as np
    cfg = _cfg(device=7 if os.environ.get("CUDA_VISIBLE_DEVICES") is None else 0)
    try:
        import torch
        if torch.cuda.is_available():
            cfg = _cfg(device=torch.cuda.device_count())
    except Exception:
        pass
    with pytest.raises(R.Rt3dError) as e:
        R.rt3d_create(cfg, np.ones(5), 2)
    assert e.value.status in (R.RT3D_E_CUDA, R.RT3D_E_INVALID)


def test_bad_irf_is_rejected_before_any_device_call(L):
    import numpy as np
    for samples, origin in ((np.ones(5), 5), (np.zeros(5), 1), (-np.ones(3), 0), (np.ones(300), 0)):
        with pytest.raises(R.Rt3dError) as e:
            R.rt3d_create(_cfg(), samples, origin)
        assert e.value.status == R.RT3D_E_INVALID


def test_workspace_bytes_and_memory_budget(L):
    """rt3d_workspace_bytes: 16 + 9K bytes per pixel of the batch plus 4 per
    sparse entry (and the call record); with max_entries = 0 a budget sets the
    entry capacity to the largest that fits; a budget below the per-pixel
    state, or below an explicit entry capacity, is refused."""
    cfg = _cfg()
    full, ent = R.workspace_bytes(cfg)
    stride = cfg.max_batch * cfg.max_h * cfg.max_w
    assert ent == stride * cfg.max_t
    fixed = full - 4 * ent
    assert fixed >= stride * (16 + 9 * cfg.k_max) and fixed < stride * (16 + 9 * cfg.k_max) + (1 << 20)
    budget = fixed + 4 * 100_000 + 3
    b, e = R.workspace_bytes(_cfg(mem_budget=budget))
    assert e == 100_000 and b <= budget
    for bad in (_cfg(mem_budget=fixed // 2), _cfg(mem_budget=budget, max_entries=200_000)):
        with pytest.raises(R.Rt3dError) as err:
            R.workspace_bytes(bad)
        assert err.value.status == R.RT3D_E_NOMEM
    with pytest.raises(R.Rt3dError) as err:
        R.workspace_bytes(_cfg(mem_budget=-1))
    assert err.value.status == R.RT3D_E_INVALID
