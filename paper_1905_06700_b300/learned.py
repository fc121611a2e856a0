"""Learned depth denoiser: training pairs from the plain method, training with
the library's own kernels, and checkpoints.

Host orchestration only: features, network passes, losses and AdamW steps run
in the library (rt3d_net_*), the plain method's steps in its loop kernels
(rt3d_phase).  A training pair is taken at every PALM iteration of a frame:
the features of the point cloud after the depth gradient step (the input the
depth denoiser sees) and a target move, divided by the depth scale, on the
alive points of the first two slots.  The target is the move to the nearest
true surface of the pixel (synthetic scenes know it) on the points within
`inlier` bins of one, or, without the scene's truth, the move the APSS
denoiser makes (a network trained so imitates APSS and cannot do better).

Checkpoint format: `<path>` holds the RT3D_NET_PARAMS float32 parameters
(little endian, the library's flat order), `<path>.json` a header with the
layer shapes, the depth scale the network was trained with and a SHA-256 of
the parameter bytes.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import rt3d as R

LAYERS = [(6, 48), (48, 48), (48, 48), (48, 2)]


def init_params(seed: int = 0) -> np.ndarray:
    """He-scaled random weights, zero biases; the last layer starts small so
    that an untrained network proposes small moves."""
    rng = np.random.default_rng(seed)
    out = []
    for l, (ci, co) in enumerate(LAYERS):
        std = np.sqrt(2.0 / (9 * ci)) * (0.1 if l == len(LAYERS) - 1 else 1.0)
        out.append(rng.normal(0.0, std, co * ci * 9))
        out.append(np.zeros(co))
    theta = np.concatenate(out).astype(np.float32)
    assert theta.size == R.NET_PARAMS
    return theta


def frame_pairs(ctx: "R.Context", net: "R.Net", dense, params: dict,
                keep: Optional[Sequence[int]] = None, truth: Optional[np.ndarray] = None,
                inlier: Optional[float] = None) -> List[Tuple]:
    """(x [1][6][h][w], target [1][2][h][w], mask [1][2][h][w]) for every
    iteration of the plain method (APSS depth denoiser) on one dense frame
    (or the iterations listed in `keep`).  With `truth` (the scene's true
    depths [S][h][w], NaN where a surface is absent) the target is the move to
    the nearest true surface, masked to the points within `inlier` bins of it;
    without, the APSS move on every alive point."""
    torch = ctx.torch
    prm = dict(params, depth_denoiser=1, warm_start=0)   # the plain method: APSS
    h, w, t = dense.shape
    scale = float(prm["net_scale"])
    csr = ctx.compact(dense)
    st = ctx.init(prm, dense=dense)
    K = int(prm["k_max"])
    tru = None
    if truth is not None:
        if inlier is None:
            raise ValueError("a truth target needs the inlier band")
        tru = torch.from_numpy(np.where(np.isfinite(truth), truth, 1e9).astype(np.float32)).to(ctx.device)
    pairs = []
    for it in range(int(prm["n_iter"])):
        ctx.phase(0, 1 if it == 0 else 0, prm, csr, st, shape=(h, w, t))
        t_half = st["t"].clone()
        x = net.features(st["t"][None], st["r"][None], st["alive"][None], scale)
        alive = st["alive"].clone()
        ctx.phase(1, 0, prm, csr, st, shape=(h, w, t))
        target = torch.zeros((1, 2, h, w), dtype=torch.float32, device=ctx.device)
        mask = torch.zeros((1, 2, h, w), dtype=torch.uint8, device=ctx.device)
        for k in range(min(K, 2)):
            if tru is None:
                target[0, k] = (st["t"][k] - t_half[k]) / scale
                mask[0, k] = alive[k]
            else:
                diff = tru - t_half[k][None]
                near = torch.gather(diff, 0, diff.abs().argmin(0, keepdim=True))[0]
                mask[0, k] = ((near.abs() < inlier) & (alive[k] > 0)).to(torch.uint8)
                target[0, k] = near / scale
        target *= mask
        if keep is None or it in keep:
            pairs.append((x, target, mask))
        ctx.phase(2, 0, prm, csr, st, shape=(h, w, t))
    torch.cuda.current_stream().synchronize()
    return pairs


def train(net: "R.Net", pairs: Sequence[Tuple], steps: int, batch: int = 8, lr: float = 1e-3,
          weight_decay: float = 1e-4, seed: int = 0, lr_final: Optional[float] = None) -> np.ndarray:
    """AdamW steps on random mini-batches of same-sized pairs; cosine decay of
    the learning rate to lr_final.  Returns the per-step losses."""
    import torch
    rng = np.random.default_rng(seed)
    lr_final = lr * 0.1 if lr_final is None else lr_final
    loss = torch.zeros(steps, dtype=torch.float32, device=pairs[0][0].device)
    for s in range(steps):
        idx = rng.integers(0, len(pairs), batch)
        x = torch.cat([pairs[i][0] for i in idx])
        tg = torch.cat([pairs[i][1] for i in idx])
        m = torch.cat([pairs[i][2] for i in idx])
        cur = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * s / max(1, steps)))
        net.train_step(x, tg, m, lr=cur, weight_decay=weight_decay, loss=loss[s:s + 1])
    return loss.cpu().numpy()


def depth_errors(result: dict, truth_depth: np.ndarray, inlier: float) -> Tuple[float, float, int]:
    """Error of the alive points against the nearest true surface of their
    pixel (truth_depth [S][h][w], NaN where a surface is absent): the RMSE
    (bins) over the points within `inlier` bins of a surface, the fraction of
    points that are, and the number of points."""
    t = result["t"].cpu().numpy().astype(np.float64)
    a = result["alive"].cpu().numpy().astype(bool)
    tru = np.where(np.isfinite(truth_depth), truth_depth, np.inf)
    err = np.min(np.abs(t[:, None] - tru[None]), axis=1)[a]
    ok = err < inlier
    rmse = float(np.sqrt(np.mean(err[ok] ** 2))) if ok.any() else 0.0
    return rmse, float(ok.mean()) if err.size else 0.0, int(err.size)


def save(path: str, theta: np.ndarray, meta: Optional[Dict] = None) -> None:
    theta = np.ascontiguousarray(np.asarray(theta, "<f4"))
    assert theta.size == R.NET_PARAMS
    raw = theta.tobytes()
    with open(path, "wb") as f:
        f.write(raw)
    head = dict(format="rt3d-learned-depth-v1", params=int(theta.size), layers=LAYERS,
                sha256=hashlib.sha256(raw).hexdigest())
    head.update(meta or {})
    with open(path + ".json", "w") as f:
        json.dump(head, f, indent=1)


def load(path: str) -> Tuple[np.ndarray, Dict]:
    with open(path + ".json") as f:
        head = json.load(f)
    with open(path, "rb") as f:
        raw = f.read()
    if head.get("format") != "rt3d-learned-depth-v1" or len(raw) != 4 * R.NET_PARAMS:
        raise ValueError(f"{path}: not a learned-depth checkpoint")
    if hashlib.sha256(raw).hexdigest() != head.get("sha256"):
        raise ValueError(f"{path}: parameter bytes do not match the header")
    return np.frombuffer(raw, "<f4").copy(), head
