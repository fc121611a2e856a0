#!/usr/bin/env python
"""Small, fixed workloads for kernel profiles (ncu captures of one launch).

Each case builds its inputs on the device, runs two warm-up calls and then
the call to capture, so `ncu -k <kernel> -s <warm-up launches> -c 1` picks a
steady-state launch.  Cases:
  init-tc       one 256x256x4096 two-surface frame at SBR 0.1, tensor-core
                (FP16) initialisation only
  init-int      the same frame, CUDA-core initialisation only
  learned       8 frames of 256x256x2048 random shapes, two PALM iterations
                with the learned depth denoiser (the committed checkpoint)
  loop          4 frames of 141x141x4096 (the benchmark scene), 20 iterations
  loop16        16 frames of the benchmark scene (the benchmark's batch; two
                chains of 8 frames each), 20 iterations
  net-forward   three forward passes of the committed network over 8 images
                of 256x256 random features (the register-staged convolution
                of the network's own training calls)

Usage: python profile_cases.py CASE
"""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import scenes  # noqa: E402
from paper_1905_06700_b300 import build as B  # noqa: E402
from paper_1905_06700_b300 import learned  # noqa: E402
from paper_1905_06700_b300 import rt3d as R  # noqa: E402

WEIGHTS = os.path.join(ROOT, "paper_1905_06700_b300", "weights", "learned_depth.bin")


def case(name: str):
    import torch
    if name == "net-forward":
        B.build()
        theta, _ = learned.load(WEIGHTS)
        net = R.Net(8, 256, 256)
        net.set_params(theta)
        x = torch.randn((8, 6, 256, 256), generator=torch.Generator().manual_seed(0)).cuda()
        for _ in range(3):
            net.forward(x)
        torch.cuda.synchronize()
        print(name, "done")
        return 0
    if name in ("init-tc", "init-int"):
        base = scenes.two_layer()
        prm = dict(scenes.make_params(base), n_iter=0, lmf_precision=2 if name == "init-tc" else 0)
        nb, mk = 1, (lambda f: scenes.two_layer(seed=1 + f))
    elif name == "learned":
        base = scenes.random_shapes(256, 256, 2048, seed=0)
        prm = dict(scenes.make_params(base), n_iter=2, depth_denoiser=2)
        nb, mk = 8, (lambda f: scenes.random_shapes(256, 256, 2048, seed=200000 + f))
    elif name in ("loop", "loop16"):
        base = scenes.net_object_wall()
        prm = scenes.make_params(base)
        nb, mk = (4 if name == "loop" else 16), (lambda f: scenes.net_object_wall(seed=1 + f))
    else:
        raise SystemExit(f"unknown case {name!r}")
    B.build()
    ctx = R.Context(base.h, base.w, base.t, prm["k_max"], base.irf.samples, base.irf.origin, max_batch=nb)
    net = None
    if prm.get("depth_denoiser") == 2:
        theta, _ = learned.load(WEIGHTS)
        net = R.Net(1, base.h, base.w)
        net.set_params(theta)
        ctx.set_depth_net(net)
    frames = [dict(dense=ctx.synthesize(scenes.sampling_tables(mk(f)))) for f in range(nb)]
    outs = [ctx.new_result(base.h, base.w, prm["k_max"]) for _ in range(nb)]
    for _ in range(3):
        ctx.reconstruct_batch(prm, frames, outs)
    torch.cuda.synchronize()
    status = ctx.device_status()
    print(name, "status", status)
    return status


if __name__ == "__main__":
    sys.exit(0 if case(sys.argv[1] if len(sys.argv) > 1 else "init-tc") == 0 else 1)
