#!/usr/bin/env python
"""Train the learned depth denoiser on the GPU and write a checkpoint.

Scenes: seeded random planes, spheres and boxes (at most two surfaces per
pixel, 1-20 signal photons per pixel, SBR 0.05-2, Gaussian IRF sigma 3 bins),
256 x 256 pixels x 2048 bins by default.  For each training scene the plain
method runs on the device and a pair (features before the depth denoiser, the
APSS move: a target from the plain method's output) is kept at a few
iterations; the network is then trained with the library's own kernels (masked
MSE, AdamW, cosine learning-rate decay).  `--target truth` takes instead the
move to the nearest true surface of the synthetic scene, on the points within
the inlier band of one.  The
held-out scenes report the inlier depth RMSE against the true surfaces for no
depth denoiser, APSS and the learned form; the report goes into the
checkpoint header.

Usage: python paper_1905_06700_b300/train_denoiser.py [--scenes 2000] [--out PATH]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import scenes  # noqa: E402
from paper_1905_06700_b300 import build as B  # noqa: E402
from paper_1905_06700_b300 import learned  # noqa: E402
from paper_1905_06700_b300 import rt3d as R  # noqa: E402

DEFAULT_OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "learned_depth.bin")


def evaluate(ctx, prm, h, w, t, seeds, inlier):
    res = {"none": [], "apss": [], "learned": []}
    for s in seeds:
        sc = scenes.random_shapes(h, w, t, seed=s)
        d = ctx.synthesize(scenes.sampling_tables(sc))
        for name, den in (("none", 0), ("apss", 1), ("learned", 2)):
            out = ctx.reconstruct(dict(prm, depth_denoiser=den), dense=d)
            res[name].append(learned.depth_errors(out, sc.depth, inlier))
    return {k: {"inlier_rmse_bins": float(np.mean([r[0] for r in v])),
                "inlier_fraction": float(np.mean([r[1] for r in v]))} for k, v in res.items()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scenes", type=int, default=2000)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--bins", type=int, default=2048)
    ap.add_argument("--keep", type=str, default="0,2,5,10,15", help="iterations whose pairs are kept")
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--target", choices=["apss", "truth"], default="apss")
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--weight-decay", type=float, default=1e-4)
    ap.add_argument("--validate", type=int, default=16)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args()
    import torch
    B.build()
    h = w = args.size
    t = args.bins
    base = scenes.random_shapes(h, w, t, seed=0)
    prm = scenes.make_params(base)
    keep = [int(v) for v in args.keep.split(",")]
    inlier = 5.0 * float(np.sqrt(base.irf.variance()))
    ctx = R.Context(h, w, t, prm["k_max"], base.irf.samples, base.irf.origin)
    net = R.Net(args.batch, h, w)
    t0 = time.time()
    pairs = []
    for s in range(args.scenes):
        sc = scenes.random_shapes(h, w, t, seed=s)
        d = ctx.synthesize(scenes.sampling_tables(sc))
        pairs += learned.frame_pairs(ctx, net, d, prm, keep=keep,
                                     truth=sc.depth if args.target == "truth" else None, inlier=inlier)
    t_pairs = time.time() - t0
    net.set_params(learned.init_params(args.seed))
    t0 = time.time()
    losses = learned.train(net, pairs, steps=args.steps, batch=args.batch, lr=args.lr,
                           weight_decay=args.weight_decay, seed=args.seed)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    del pairs
    ctx.set_depth_net(net)
    report = evaluate(ctx, prm, h, w, t, range(100000, 100000 + args.validate), inlier)
    theta = net.get_params()
    meta = dict(trained_on=dict(generator="random_shapes", scenes=args.scenes, size=[h, w, t],
                                iterations_kept=keep, seeds=[0, args.scenes - 1], target=args.target,
                                inlier_bins=inlier),
                training=dict(steps=args.steps, batch=args.batch, lr=args.lr, weight_decay=args.weight_decay,
                              loss_first=float(losses[:50].mean()), loss_last=float(losses[-50:].mean()),
                              seconds_pairs=round(t_pairs, 1), seconds_train=round(t_train, 1)),
                net_scale=float(prm["net_scale"]), net_fallback=float(prm["net_fallback"]),
                validation=dict(scenes=args.validate, seeds=[100000, 100000 + args.validate - 1],
                                inlier_bins=inlier, **report))
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    learned.save(args.out, theta, meta)
    print(json.dumps(meta, indent=1))


if __name__ == "__main__":
    main()
