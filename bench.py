#!/usr/bin/env python
"""Throughput and latency of the full reconstruction on one B300.

Workload: the multi-surface scene at 141 x 141 pixels x 4096 bins (a
camouflage-like net at bin 1500, a smooth object at 1800-2200, a wall at
3000; gamma IRF of shape 3 and scale 5 bins; 5 signal photons per pixel at a
signal-to-background ratio of 1), synthesised on the device from seeded
Philox draws.  One step = the whole method (initialisation + 20 PALM
iterations) on a batch of frames, inputs resident in HBM; the batch's dense
histograms (2.6 GB for 16 frames) exceed the 126 MB L2, so every step streams
its inputs from HBM.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B]
                       [--impl ours|reference]
Multi-GPU (torchrun, one rank per GPU): independent replicas, no collective
on the data path; value = all frames / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import scenes  # noqa: E402

METRIC = "frames/s (141x141 px x 4096 bins, multi-surface, full method)"
UNIT = "frames/s"
H, W, T, K = 141, 141, 4096, 3
KERNEL_NAMES = ["init", "phase_a", "phase_b", "phase_c", "final"]
WEIGHTS = os.path.join(ROOT, "paper_1905_06700_b300", "weights", "learned_depth.bin")
# the same network trained toward the synthetic scenes' true surfaces instead
# of the plain method's output (reported beside the default checkpoint)
WEIGHTS_TRUTH = os.path.join(ROOT, "paper_1905_06700_b300", "weights", "learned_depth_truth.bin")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--latency-frames", type=int, default=128)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-frames", type=int, default=4)
    ap.add_argument("--cpu-single-frames", type=int, default=1,
                    help="frames of the single-thread oracle timing (0 = skip)")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="duration of the continuous-batching serving run at 500 frames/s (0 = skip; "
                         "the learned form runs up to 20 s, the overload run up to 8 s)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the precision (tensor-core init) and learned forms")
    ap.add_argument("--form-steps", type=int, default=5)
    ap.add_argument("--no-sweep", dest="sweep", action="store_false",
                    help="skip the execution-time sweeps over pixels and active bins (Fig. 5)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# --------------------------------------------------------------------------- helpers

def replica_seeds(rank: int, frames: int) -> list:
    """Scene seeds of one replica: every rank reconstructs different frames."""
    return [1 + rank * frames + f for f in range(frames)]


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The slowest rank's time (the job's time); no collective on one GPU."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(frames_per_rank_step: int, steps: int, world: int, t_max_ms: float) -> float:
    """Whole-job frames/s: all ranks' frames over the slowest rank's time."""
    return frames_per_rank_step * steps * world / (t_max_ms / 1000.0)


def algorithmic_bytes(n_px: int, t: int, nnz_total: int, k: int, fused_frac: float = 0.0) -> dict:
    """Bytes each kernel class must move per launch for n_px pixels of T bins
    (every array read or written once; halos counted once).  Per pixel:
      init    2T dense read + 8 seg + 9K state + 4 b written, + 4 per nonzero entry written
      phase A 8 seg + 4 b_half + K (4 t + 4 r + 1 alive_b + 1 alive + 4 t_half) + 4 b, + 4/entry
      phase B 8 seg + K (4 t_half + 1 alive + 4 r + 4 t + 4 r_half) + 4 b, + 4/entry
      phase C 8 seg + K (4 t + 4 r_half + 1 alive + 4 r + 1 alive_b) + 4 b + 4 b_half, + 4/entry;
              a launch that also runs the next iteration's depth step (fused_frac of
              them) writes K x 4 t_half + 4 b more
      final   K (1 alive_b + 1 alive) + 4 b_half + 4 b."""
    px = n_px
    e = 4 * nnz_total
    return {
        "init": px * (2 * t + 8 + 9 * k + 4) + e,
        "phase_a": px * (8 + 4 + k * 14 + 4) + e,
        "phase_b": px * (8 + k * 17 + 4) + e,
        "phase_c": px * (8 + k * 14 + 8) + e + fused_frac * px * (4 * k + 4),
        "final": px * (2 * k + 8),
    }


LOOP_KERNELS = ("phase_a", "phase_b", "phase_c", "final")


def loop_bytes_per_call(n_px: int, t: int, nnz_total: int, k: int, prm) -> float:
    """Algorithmic bytes of a call's whole PALM loop (every launch of phases
    A, B, C and the finaliser), from the per-launch table above and the
    launch counts the library makes: with the identity background denoiser
    one phase A, then n_iter x (B, C) with all but the last C also running
    the next depth step; otherwise n_iter x (A, B, C); one finaliser."""
    n = int(prm["n_iter"])
    if n <= 0:
        return 0.0
    a = algorithmic_bytes(n_px, t, nnz_total, k, fused_fraction(prm))
    n_a = n if prm.get("bkg_mode", 0) == 1 else 1
    return n_a * a["phase_a"] + n * (a["phase_b"] + a["phase_c"]) + a["final"]


def method_work(outs, nnz_px, prm, k):
    """The FP32 work the method itself needs in one APSS + intensity-step pass
    (phase B), counted on the final point clouds of the call's frames:
      per alive point, per alive candidate in the window cells inside the
      lateral radius: a distance test (4 FLOP: difference, scale, square-add,
      compare);
      per neighbour inside the 3-D radius: the weight and the 14 moment sums
      (30 FLOP);
      per point with a fit: the centred 3x3 solve and projection (60 FLOP);
      the intensity step's bin sums: per nonzero bin and alive point of its
      pixel, the cubic IRF value and slope, the point's share of lambda and the
      sum (15 FLOP), and per bin lambda and its reciprocal (3 FLOP).
    Returns (flop, counts)."""
    R, pitch, hr = int(prm["win_r"]), float(prm["pixel_pitch"]), float(prm["apss_radius"])
    cells = [(di, dj) for di in range(-R, R + 1) for dj in range(-R, R + 1)
             if (pitch * di / hr) ** 2 + (pitch * dj / hr) ** 2 < 1.0]
    tests = inwin = pts = 0
    bin_slots = 0
    for o, nz in zip(outs, nnz_px):
        t = o["t"].cpu().numpy().astype(np.float64)
        a = o["alive"].cpu().numpy().astype(bool)
        kk, hh, ww = t.shape
        pts += int(a.sum())
        bin_slots += int((nz * a.sum(0)).sum())
        for di, dj in cells:
            i0, i1 = max(0, -di), min(hh, hh - di)
            j0, j1 = max(0, -dj), min(ww, ww - dj)
            if i0 >= i1 or j0 >= j1:
                continue
            r2 = (pitch * di / hr) ** 2 + (pitch * dj / hr) ** 2
            for n in range(kk):
                an = a[n, i0:i1, j0:j1]
                tn = t[n, i0:i1, j0:j1]
                for m in range(kk):
                    am = a[m, i0 + di:i1 + di, j0 + dj:j1 + dj]
                    both = an & am
                    tests += int(both.sum())
                    z = (t[m, i0 + di:i1 + di, j0 + dj:j1 + dj] - tn) / hr
                    inwin += int((both & (r2 + z * z < 1.0)).sum())
    nnz_total = int(sum(int(x.sum()) for x in nnz_px))
    flop = 4 * tests + 30 * inwin + 60 * pts + 15 * bin_slots + 3 * nnz_total
    return flop, {"alive_points": pts, "candidate_tests": tests, "in_window_neighbours": inwin,
                  "nonzero_bins": nnz_total, "bin_point_pairs": bin_slots,
                  "tests_per_point": round(tests / max(pts, 1), 2),
                  "neighbours_per_point": round(inwin / max(pts, 1), 2)}


def fused_fraction(prm) -> float:
    """Share of phase C launches that also run the next iteration's depth step
    (the library fuses it when the background denoiser is the identity): all
    but the last iteration's."""
    n = int(prm["n_iter"])
    if n <= 0 or prm.get("bkg_mode", 0) == 1:
        return 0.0
    return (n - 1) / n


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                mhz.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(mhz) if mhz else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(mhz)}


def measured_peaks() -> dict:
    """HBM copy bandwidth (measured) and the FP32 FMA peak derived from the unit
    counts: 148 SMs x 128 FP32 lanes x 2 FLOP x the maximum SM clock."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    d = json.load(open(path)) if os.path.exists(path) else {}
    mhz = d.get("sm_max_mhz", 2032.0)
    return {"hbm_gbs": d.get("hbm_gbs", 6400.0), "source": "measured" if d else "fallback",
            "fp32_tflops": 148 * 128 * 2 * mhz * 1e6 / 1e12}


def traffic_record(kernel: str):
    """dram bytes per launch of `kernel` from the committed ncu summary, or None
    if the kernel sources changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec:
        return None
    from paper_1905_06700_b300 import build as B
    if rec.get("sources_sha") != B.sources_sha():
        return None
    return rec.get("dram_bytes_per_launch_full")


def bench_config(world: int) -> dict:
    """The workload both arms name (the reference arm runs a bounded sample of it)."""
    return {"workload": "net_object_wall 141x141x4096, K=3, gamma IRF (3,5), "
                        "5 signal photons/px, SBR 1, 20 PALM iterations",
            "l2": "inputs larger than L2 (dense histograms stream from HBM each step)",
            "parallelism": f"replicas x{world}"}


# --------------------------------------------------------------------------- our arm

def run_ours(args, world, rank, local):
    import torch
    from paper_1905_06700_b300 import build as B
    from paper_1905_06700_b300 import rt3d as R
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    nb = args.batch
    base = scenes.net_object_wall(H, W, T)
    prm = scenes.make_params(base)
    assert prm["k_max"] == K
    ctx = R.Context(H, W, T, K, base.irf.samples, base.irf.origin, max_batch=nb, device=local)
    dense = []
    seeds = replica_seeds(rank, nb)
    for seed in seeds:
        sc = scenes.net_object_wall(H, W, T, seed=seed)
        dense.append(ctx.synthesize(scenes.sampling_tables(sc)))
    torch.cuda.synchronize()
    nnz_total = int(sum(int(torch.count_nonzero(d.view(torch.int16)).item()) for d in dense))
    frames = [dict(dense=d) for d in dense]
    outs = [ctx.new_result(H, W, K) for _ in range(nb)]
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        ctx.reconstruct_batch(prm, frames, outs)
    torch.cuda.synchronize()
    assert ctx.device_status() == R.RT3D_OK

    # ---------------- timed region (no per-kernel events: the library runs
    # the batch as two parallel chains of frames)
    launches0 = ctx.launch_count()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    evs[0].record(stream)
    for i in range(args.steps):
        ctx.reconstruct_batch(prm, frames, outs)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = ctx.launch_count() - launches0
    ms_total = evs[0].elapsed_time(evs[-1])
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    assert ctx.device_status() == R.RT3D_OK

    # ---------------- per-kernel durations (CUDA events around every launch;
    # with events the library keeps one chain, so each kernel runs alone)
    ctx.set_profiling(True)
    ctx.reconstruct_batch(prm, frames, outs)          # capture of the timed graph
    torch.cuda.synchronize()
    ctx.kernel_times(reset=True)
    for _ in range(max(2, min(args.steps, 5))):
        ctx.reconstruct_batch(prm, frames, outs)
    torch.cuda.synchronize()
    ktimes = ctx.kernel_times(reset=True)
    ctx.set_profiling(False)
    assert ctx.device_status() == R.RT3D_OK

    t_max = max_over_ranks(ms_total, world, dev)
    value = job_throughput(nb, args.steps, world, t_max)

    # ---------------- the loop's own time: the same two-chain call with no
    # PALM iteration (initialisation and finaliser only), subtracted
    outs0 = [ctx.new_result(H, W, K) for _ in range(nb)]
    ms_init_only = time_calls(ctx, dict(prm, n_iter=0), frames, outs0, max(3, min(args.steps, 10)))
    del outs0
    ms_loop = ms_total / args.steps - ms_init_only

    # ---------------- rooflines (the path is HBM-bound: algorithmic bytes per launch / time)
    n_px = nb * H * W
    ff = fused_fraction(prm)
    alg = algorithmic_bytes(n_px, T, nnz_total, K, ff)
    peaks = measured_peaks()
    per_kernel = {}
    for name in KERNEL_NAMES:
        ms, n = ktimes[name]
        if n:
            sec = ms / n / 1000.0
            per_kernel[name] = dict(ms_total=ms, launches=n, ms_per_launch=ms / n,
                                    alg_bytes_per_launch=alg[name], gbs=alg[name] / sec / 1e9,
                                    hbm_frac=alg[name] / sec / 1e9 / peaks["hbm_gbs"])
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms_total"])
    d = per_kernel[dom]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(d["gbs"], 1),
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(d["hbm_frac"], 4),
                "peak_source": f"{peaks['source']} copy bandwidth (burst), of {peaks['source']}",
                "alg_bytes_per_launch": int(d["alg_bytes_per_launch"]),
                "ms_per_launch": round(d["ms_per_launch"], 5),
                "traffic": traffic_record(dom)}
    lb = loop_bytes_per_call(n_px, T, nnz_total, K, prm)
    loop_roofline = {"bound": "hbm", "what": "all PALM-loop launches of a call (phases A, B, C, finaliser)",
                     "alg_bytes_per_step": int(lb), "loop_ms_per_step": round(ms_loop, 4),
                     "step_ms_without_iterations": round(ms_init_only, 4),
                     "achieved": round(lb / (ms_loop * 1e-3) / 1e9, 1), "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": round(lb / (ms_loop * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                     "method": "loop time = two-chain step time minus the same call with n_iter = 0"}
    # the ALU view of the dominant loop kernel, counting only the method's work
    nnz_px = [torch.count_nonzero(dd.view(torch.int16), dim=2).cpu().numpy() for dd in dense]
    flop_b, work = method_work(outs, nnz_px, prm, K)
    alu_view = None
    if "phase_b" in per_kernel:
        sec_b = per_kernel["phase_b"]["ms_per_launch"] * 1e-3
        alu_view = {"bound": "alu", "kernel": "phase_b", "alg_flop_per_launch": int(flop_b),
                    "achieved": round(flop_b / sec_b / 1e12, 3), "peak": round(peaks["fp32_tflops"], 1),
                    "unit": "TFLOP/s", "frac": round(flop_b / sec_b / 1e12 / peaks["fp32_tflops"], 4),
                    "peak_source": "FP32 FMA: 148 SMs x 128 lanes x 2 x max SM clock",
                    "work_counted_on_final_state": work}

    result = None
    if rank == 0:
        # ---------------- single-frame latency (batch of one)
        lat = []
        one = ctx.new_result(H, W, K)
        for i in range(args.latency_frames + 3 if args.latency_frames > 0 else 0):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.reconstruct(prm, dense=dense[i % nb], out=one)
            b.record(stream)
            b.synchronize()
            if i >= 3:
                lat.append(a.elapsed_time(b))
        lat.sort()
        if not lat:
            lat = [float("nan")]

        # ---------------- end to end through the host entry point
        e2e_forms = run_e2e(args, ctx, prm, dense, R) if args.e2e_steps > 0 else None
        e2e = e2e_forms["dense"] if e2e_forms else None
        e2e_sparse = e2e_forms["sparse"] if e2e_forms else None

        # ---------------- the oracle on the host cores (and, there, the parity
        # of the benchmark's first frame against it)
        cpu, parity = None, None
        if world == 1 and args.cpu_frames >= 1:
            cpu, parity = cpu_baseline(args, prm, None if args.no_parity else (seeds[0], outs[0]))

        # ---------------- continuous-batching serving of mixed streams
        serving = None
        if args.serve_seconds > 0:
            serving = {"plain": run_serving(args, local),
                       # offered above capacity: batches fill, throughput is the capacity
                       "plain_overload": run_serving(args, local, rate_hz=6000.0,
                                                     seconds=min(args.serve_seconds, 8.0))}
            if not args.no_forms:
                serving["learned"] = run_serving(args, local, learned_form=True,
                                                 seconds=min(args.serve_seconds, 20.0))

        # ---------------- execution time against pixels and active bins (Fig. 5)
        sweep = run_fig5_sweep(args, local) if args.sweep else None

        # ---------------- the precision and learned forms
        forms = None
        if not args.no_forms:
            forms = {"tensor_core_init_on_this_workload": run_tc_headline(args, ctx, prm, frames, outs, peaks),
                     "precision": run_precision_form(args, local, peaks, with_oracle=not args.no_parity),
                     "learned": run_learned_form(args, local, with_oracle=not args.no_parity),
                     "super_resolution": run_super_resolution(args, local)}

        result = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (matched filter int32)", "data": "synthetic (seeded Philox, device-resident)",
            "config": bench_config(world),
            "frames_per_step": nb, "nnz_per_pixel": round(nnz_total / (nb * H * W), 2),
            "latency_ms": {"batch_step_p50": round(statistics.median(step_ms), 4),
                           "batch_step_p99": round(float(np.percentile(step_ms, 99)), 4),
                           "frame_p50": round(float(np.percentile(lat, 50)), 4),
                           "frame_p99": round(float(np.percentile(lat, 99)), 4),
                           "frame_samples": len(lat)},
            "e2e": e2e,
            "e2e_sparse": e2e_sparse,
            "roofline": roofline,
            "loop_roofline": loop_roofline,
            "alu_view": alu_view,
            "init_roofline": {"bound": "hbm", "achieved": round(per_kernel["init"]["gbs"], 1),
                              "peak": peaks["hbm_gbs"], "unit": "GB/s",
                              "frac": round(per_kernel["init"]["hbm_frac"], 4),
                              "traffic": traffic_record("init")} if "init" in per_kernel else None,
            "kernels": {k: {kk: round(vv, 4) if isinstance(vv, float) else vv for kk, vv in v.items()}
                        for k, v in per_kernel.items()},
            "gpu_launches": int(launches),
            "clocks": clk,
            "parity": parity,
            "serving": serving,
            "forms": forms,
            "fig5_sweep": sweep,
            "cpu_baseline": cpu,
        }
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    ctx.close()
    return result


def time_steps(ctx, prm, frames, outs, steps, warmup=2):
    """Mean ms per batched call (no per-kernel events, as a caller runs it) and
    mean ms per launch of each kernel class (a separate run with events around
    every launch, where each kernel runs alone)."""
    import torch
    for _ in range(warmup):
        ctx.reconstruct_batch(prm, frames, outs)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        ctx.reconstruct_batch(prm, frames, outs)
    b.record()
    b.synchronize()
    ctx.set_profiling(True)
    ctx.reconstruct_batch(prm, frames, outs)
    torch.cuda.synchronize()
    ctx.kernel_times(reset=True)
    for _ in range(steps):
        ctx.reconstruct_batch(prm, frames, outs)
    torch.cuda.synchronize()
    kt = ctx.kernel_times(reset=True)
    ctx.set_profiling(False)
    return a.elapsed_time(b) / steps, {k: v[0] / v[1] for k, v in kt.items() if v[1]}


def time_calls(ctx, prm, frames, outs, steps, warmup=2):
    """Mean ms per batched call, timed with CUDA events on the current stream
    (no per-kernel events: the library's production two-chain graph)."""
    import torch
    for _ in range(warmup):
        ctx.reconstruct_batch(prm, frames, outs)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        ctx.reconstruct_batch(prm, frames, outs)
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / steps


def init_bytes(n_px, t, k, nnz_total):
    """Algorithmic bytes of the initialisation (see algorithmic_bytes)."""
    return n_px * (2 * t + 8 + 9 * k + 4) + 4 * nnz_total


def run_tc_headline(args, ctx, prm, frames, outs, peaks) -> dict:
    """The tensor-core initialisation (FP16 and BF16 operands) on the benchmark
    workload; results must equal the integer path's bit for bit."""
    import torch
    ref = [{k: v.clone() for k, v in o.items()} for o in outs]
    nb = len(frames)
    nnz = int(sum(int(torch.count_nonzero(f["dense"].view(torch.int16)).item()) for f in frames))
    out = {}
    for name, mode in (("fp16", 2), ("bf16", 1)):
        ms, kt = time_steps(ctx, dict(prm, lmf_precision=mode), frames, outs, args.form_steps)
        same = all(torch.equal(a[k], b[k]) for a, b in zip(ref, outs) for k in ("t", "r", "alive", "b"))
        ib = init_bytes(nb * H * W, T, K, nnz)
        gbs = ib / (kt["init_tc"] * 1e-3) / 1e9
        out[name] = {"frames_per_s": round(nb / (ms / 1000), 2), "init_tc_ms": round(kt["init_tc"], 4),
                     "init_gbs": round(gbs, 1), "init_hbm_frac": round(gbs / peaks["hbm_gbs"], 4),
                     "bitwise_equal_to_integer_path": bool(same)}
    for o, r in zip(outs, ref):
        for k in o:
            o[k].copy_(r[k])
    return out


def run_precision_form(args, device, peaks, with_oracle=True) -> dict:
    """Precision form: 256 x 256 x 4096, two surfaces, SBR 0.1 (about 54
    photons per pixel), 8 frames per step; the matched filter on CUDA cores
    (integer) and on tensor cores (FP16 and BF16 operands, FP32 accumulation).
    The filter output is an exact integer in every mode, so the results are
    bitwise equal; each mode's first frame is also compared with the FP64
    oracle (depth error max / p99.9 / fraction within 1e-3 bins).  The loop's
    HBM roofline fraction is reported for this workload too."""
    import torch
    from paper_1905_06700_b300 import rt3d as R
    h = w = 256
    t = 4096
    nb = 8
    base = scenes.two_layer(h, w, t)
    prm = scenes.make_params(base, apss_fp64=1)        # this form solves APSS in FP64
    k = prm["k_max"]
    ctx = R.Context(h, w, t, k, base.irf.samples, base.irf.origin, max_batch=nb, device=device)
    dense = [ctx.synthesize(scenes.sampling_tables(scenes.two_layer(h, w, t, seed=1 + f))) for f in range(nb)]
    torch.cuda.synchronize()
    nnz = int(sum(int(torch.count_nonzero(d.view(torch.int16)).item()) for d in dense))
    frames = [dict(dense=d) for d in dense]
    outs = [ctx.new_result(h, w, k) for _ in range(nb)]
    res = {"workload": "two_layer 256x256x4096, K=2, gamma IRF (3,5), 5 signal photons/px, SBR 0.1, "
                       "20 PALM iterations, 8 frames per step; APSS normal equations solved in FP64 "
                       "(integer_fp32_solve: the same in FP32)",
           "nnz_per_pixel": round(nnz / (nb * h * w), 1)}
    oracle_runs = {}
    if with_oracle:
        import oracle
        from oracle import compare
        oracle.build()
        z0 = dense[0].view(torch.int16).cpu().numpy().view(np.uint16)
        oirf = oracle.OIrf(base.irf.samples, base.irf.origin)
        oracle_runs = {1: compare.reconstruct_with_probes(z0, oirf, prm),
                       0: compare.reconstruct_with_probes(z0, oirf, dict(prm, apss_fp64=0))}
        # the FP64 oracle's own time on this workload (one frame, the host's cores)
        t0 = time.perf_counter()
        oracle.reconstruct(z0, oirf, prm)
        sec = time.perf_counter() - t0
        res["cpu_fp64_oracle"] = {"frames_per_s": round(1.0 / sec, 4), "cores": oracle.num_threads(), "kind": "oracle",
                                  "sample": "frame 0 of the workload (init + 20 iterations, FP64 APSS solve), OpenMP"}
    ref = None
    for name, mode, fp64 in (("integer", 0, 1), ("fp16", 2, 1), ("bf16", 1, 1), ("integer_fp32_solve", 0, 0)):
        ms, kt = time_steps(ctx, dict(prm, lmf_precision=mode, apss_fp64=fp64), frames, outs, args.form_steps)
        init_ms = kt.get("init", 0.0) + kt.get("init_tc", 0.0)
        gbs = init_bytes(nb * h * w, t, k, nnz) / (init_ms * 1e-3) / 1e9
        entry = {"frames_per_s": round(nb / (ms / 1000), 2), "init_ms": round(init_ms, 4),
                 "init_gbs": round(gbs, 1), "init_hbm_frac": round(gbs / peaks["hbm_gbs"], 4),
                 "phase_b_ms": round(kt.get("phase_b", 0.0), 4),
                 "apss_solve": "fp64" if fp64 else "fp32"}
        if ref is None:
            ref = [{kk: v.clone() for kk, v in o.items()} for o in outs]
            # the loop's HBM roofline on this workload
            ms0 = time_calls(ctx, dict(prm, n_iter=0), frames, [ctx.new_result(h, w, k) for _ in range(nb)],
                             args.form_steps)
            lb = loop_bytes_per_call(nb * h * w, t, nnz, k, prm)
            loop_ms = ms - ms0
            res["loop_roofline"] = {"bound": "hbm", "alg_bytes_per_step": int(lb),
                                    "loop_ms_per_step": round(loop_ms, 4),
                                    "achieved": round(lb / (loop_ms * 1e-3) / 1e9, 1), "unit": "GB/s",
                                    "peak": peaks["hbm_gbs"],
                                    "frac": round(lb / (loop_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}
        elif fp64:
            entry["bitwise_equal_to_integer_path"] = bool(all(
                torch.equal(a[kk], b[kk]) for a, b in zip(ref, outs) for kk in ("t", "r", "alive", "b")))
        if fp64 in oracle_runs:
            from oracle import compare
            o, probes = oracle_runs[fp64]
            g = {kk: v.cpu().numpy() for kk, v in outs[0].items() if kk != "n_points"}
            st = compare.cloud_stats(g, o, probes, t, 1e-3, 1e-4, r_min=prm["r_min"])
            entry["vs_fp64_oracle_frame0"] = {
                "points": st["points"], "alive_mismatch": st["all_alive_mismatch"],
                "dt_max_bins": st["all_dt_max"], "dt_p999_bins": st["all_dt_p999"],
                "frac_within_1e-3_bins": st["all_frac_within_tol"],
                "ill_conditioned": st["ill"], "dt_max_bins_well_conditioned": st["dt_max"],
                "dr_max_rel_well_conditioned": st["dr_max"],
                "ill_conditioned_over_3x_probe_deviation": st["ill_over_bound"],
                "ill_conditioned_worst_ratio_to_probe": st["ill_ratio_max"],
                "db_max_rel_well_conditioned": st["db_max"],
                "ill_conditioned_backgrounds": st["ill_background_pixels"],
                "ill_backgrounds_over_3x_probe_deviation": st["ill_background_over_bound"]}
        res[name] = entry
    assert ctx.device_status() == R.RT3D_OK
    ctx.close()
    return res


def learned_oracle_error(sc, dense, out, prm, theta) -> dict:
    """The learned form's error against the FP64 oracle running the same
    network on the same frame (the stated error of the bf16 form)."""
    import torch
    import oracle
    oracle.build()
    z = dense.view(torch.int16).cpu().numpy().view(np.uint16)
    o = oracle.reconstruct(z, oracle.OIrf(sc.irf.samples, sc.irf.origin),
                           dict(prm, net_theta=np.asarray(theta, np.float64)))
    g = {k: v.cpu().numpy() for k, v in out.items() if k != "n_points"}
    ga, oa = g["alive"].astype(bool), o.alive.astype(bool)
    both = ga & oa
    dt = np.abs(g["t"].astype(np.float64) - o.t)[both]
    dr = (np.abs(g["r"].astype(np.float64) - o.r) / np.maximum(o.r, 0.1))[both]
    return {"points": int(oa.sum()), "alive_mismatch": int((ga != oa).sum()),
            "dt_median_bins": float(np.median(dt)), "dt_p99_bins": float(np.percentile(dt, 99)),
            "dt_p999_bins": float(np.percentile(dt, 99.9)), "dt_max_bins": float(dt.max()),
            "frac_within_1e-3_bins": float((dt <= 1e-3).mean()),
            "dr_median_rel": float(np.median(dr)), "dr_p99_rel": float(np.percentile(dr, 99))}


def run_learned_form(args, device, with_oracle=True) -> dict:
    """Learned form and the other plug-in depth denoisers: 256 x 256 x 2048
    random planes, spheres and boxes (1-20 signal photons/px, SBR 0.05-2);
    throughput, single-frame latency and the inlier depth error against the
    true surfaces (points within 5 IRF sigma) for no depth denoiser, APSS,
    the local plane fit, the bilateral depth filter and the learned form (the
    committed network in place of APSS, trained on the plain method's output;
    and, as `learned_truth_target`, the same network trained toward the true
    surfaces)."""
    import torch
    from paper_1905_06700_b300 import learned
    from paper_1905_06700_b300 import rt3d as R
    if not os.path.exists(WEIGHTS):
        return {"unavailable": "no trained checkpoint at paper_1905_06700_b300/weights/learned_depth.bin"}
    theta, head = learned.load(WEIGHTS)
    h = w = 256
    t = 2048
    nb = 8
    base = scenes.random_shapes(h, w, t, seed=0)
    prm = scenes.make_params(base)
    k = prm["k_max"]
    ctx = R.Context(h, w, t, k, base.irf.samples, base.irf.origin, max_batch=nb, device=device)
    net = R.Net(1, h, w, device=device)
    net.set_params(theta)
    ctx.set_depth_net(net)
    scs = [scenes.random_shapes(h, w, t, seed=200000 + f) for f in range(nb)]
    dense = [ctx.synthesize(scenes.sampling_tables(sc)) for sc in scs]
    torch.cuda.synchronize()
    frames = [dict(dense=d) for d in dense]
    outs = [ctx.new_result(h, w, k) for _ in range(nb)]
    inlier = 5.0 * float(np.sqrt(base.irf.variance()))
    res = {"workload": "random_shapes 256x256x2048 (seeds 200000-200007), K=2, Gaussian IRF sigma 3, "
                       "20 PALM iterations, 8 frames per step",
           "checkpoint": {kk: head[kk] for kk in ("trained_on", "training") if kk in head}}
    forms = [("none", 0), ("apss", 1), ("plane", 3), ("bilateral", 4), ("learned", 2)]
    if os.path.exists(WEIGHTS_TRUTH):
        forms.append(("learned_truth_target", 2))
    for name, den in forms:
        if name == "learned_truth_target":
            theta_t, head_t = learned.load(WEIGHTS_TRUTH)
            net_t = R.Net(1, h, w, device=device)
            net_t.set_params(theta_t)
            ctx.set_depth_net(net_t)
        p = dict(prm, depth_denoiser=den)
        ms, kt = time_steps(ctx, p, frames, outs, args.form_steps)
        errs = [learned.depth_errors(o, sc.depth, inlier) for o, sc in zip(outs, scs)]
        lat = []
        one = ctx.new_result(h, w, k)
        for i in range(12):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.reconstruct(p, dense=dense[i % nb], out=one)
            b.record()
            b.synchronize()
            if i >= 2:
                lat.append(a.elapsed_time(b))
        if name == "learned" and with_oracle:
            res["learned_vs_fp64_oracle_frame0"] = learned_oracle_error(scs[0], dense[0], outs[0], p, theta)
        res[name] = {"frames_per_s": round(nb / (ms / 1000), 2),
                     "frame_latency_ms_p50": round(float(np.percentile(lat, 50)), 3),
                     "frame_latency_ms_p99": round(float(np.percentile(lat, 99)), 3),
                     # phase B (APSS / fallback) + features and 4 convolutions of the network
                     "depth_step_ms_per_iteration": round(kt.get("phase_b", 0.0) + 5 * kt.get("net", 0.0), 4),
                     "inlier_depth_rmse_bins": round(float(np.mean([e[0] for e in errs])), 4),
                     "inlier_fraction": round(float(np.mean([e[1] for e in errs])), 4)}
        if name == "learned_truth_target":
            res[name]["checkpoint"] = {kk: head_t[kk] for kk in ("trained_on", "training") if kk in head_t}
    assert ctx.device_status() == R.RT3D_OK
    ctx.close()
    return res


def run_fig5_sweep(args, device) -> dict:
    """Execution time per frame against (a) the pixel count at about four
    active bins per pixel and (b) the mean number of active (nonzero) bins
    per pixel at 141 x 141 pixels (Methods, Fig. 5), on head-like frames
    (one surface per pixel, two at the head's rim; gamma IRF; 3 signal
    photons per pixel, T = 4096, K = 2, 20 PALM iterations).  Per point: the
    median over repeated single-frame calls (the paper's per-frame time, CUDA
    events, inputs resident) and the per-frame time of 8-frame batched calls."""
    import torch
    from paper_1905_06700_b300 import rt3d as R
    t = 4096
    reps = 7

    def measure(h, w, bkg_photons, nb=8):
        scs = [scenes.head_like(h, w, t, seed=1 + f, bkg_photons=bkg_photons) for f in range(nb)]
        prm = scenes.make_params(scs[0])
        k = prm["k_max"]
        exp_nnz = 4.0 + bkg_photons
        ctx = R.Context(h, w, t, k, scs[0].irf.samples, scs[0].irf.origin, max_batch=nb, device=device,
                        max_entries=int(nb * h * w * (2 * exp_nnz + 64)))
        dense = [ctx.synthesize(scenes.sampling_tables(sc)) for sc in scs]
        torch.cuda.synchronize()
        nnz = float(np.mean([torch.count_nonzero(d.view(torch.int16)).item() / (h * w) for d in dense]))
        one = ctx.new_result(h, w, k)
        lat = []
        for i in range(reps + 2):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.reconstruct(prm, dense=dense[i % nb], out=one)
            b.record()
            b.synchronize()
            if i >= 2:
                lat.append(a.elapsed_time(b))
        outs = [ctx.new_result(h, w, k) for _ in range(nb)]
        ms = time_calls(ctx, prm, [dict(dense=d) for d in dense], outs, 3)
        assert ctx.device_status() == R.RT3D_OK
        ctx.close()
        del dense, outs
        torch.cuda.empty_cache()
        return {"pixels": h * w, "mean_active_bins": round(nnz, 2),
                "frame_ms_single": round(float(np.median(lat)), 4),
                "frame_ms_batched": round(ms / nb, 4)}

    by_pixels = [dict(side=sd, **measure(sd, sd, 1.2)) for sd in (32, 64, 96, 141, 192, 256, 384, 512)]
    by_bins = [dict(bkg_photons=bp, **measure(141, 141, bp)) for bp in (0.0, 1.0, 3.0, 8.0, 20.0, 50.0, 100.0, 200.0)]
    x = np.array([r["mean_active_bins"] for r in by_bins])
    y = np.array([r["frame_ms_single"] for r in by_bins])
    slope, icpt = np.polyfit(x, y, 1)
    return {"workload": "head_like frames, T=4096, K=2, gamma IRF (3,5), 3 signal photons/px, 20 iterations",
            "time_vs_pixels_4_active_bins": by_pixels,
            "time_vs_active_bins_141x141": by_bins,
            "linear_fit_single_frame_ms_vs_active_bins": {"slope_ms_per_bin": round(float(slope), 5),
                                                          "intercept_ms": round(float(icpt), 4)}}


def run_super_resolution(args, device) -> dict:
    """Super-resolution (Results, "3D Dynamic scenes"): 32 x 32 pixels x 153
    bins (~450 signal and ~450 background photons per pixel; a camouflage net,
    two people walking behind it and a backplane) reconstructed on the 96 x 96
    world grid through the point-to-cube mapping f (u = 3), K = 2, 20
    iterations, 8 frames (the people moving 1 world pixel per frame) per call;
    frames/s, single-frame latency and the depth error of the world points
    against the true world surfaces, beside the same frames without
    super-resolution (points on the 32 x 32 pixel grid)."""
    import torch
    from paper_1905_06700_b300 import rt3d as R
    h = w = 32
    t, up, nb = 153, 3, 8
    made = [scenes.camouflage_people(h, w, t, up=up, seed=1, frame=f) for f in range(nb)]
    base = made[0][0]
    ctx = R.Context(h * up, w * up, t, 2, base.irf.samples, base.irf.origin, max_batch=nb, device=device)
    dense = [ctx.synthesize(scenes.sampling_tables(sc)) for sc, _ in made]
    torch.cuda.synchronize()
    frames = [dict(dense=d) for d in dense]
    res = {"workload": "camouflage_people 32x32x153 -> 96x96 (u=3), ~900 photons/px, K=2, Gaussian IRF "
                       "sigma 1 bin, 20 PALM iterations, 8 frames per call",
           "nnz_per_pixel": round(float(np.mean([torch.count_nonzero(d.view(torch.int16)).item() / (h * w)
                                                 for d in dense])), 1)}
    for name, u, pitch in (("super_resolved", up, 4.0), ("pixel_grid", 1, 4.0 * up)):
        prm = scenes.make_params(base, pixel_pitch=pitch, k_max=2, upsample=u)
        outs = [ctx.new_result(h, w, 2, u) for _ in range(nb)]
        ms = time_calls(ctx, prm, frames, outs, args.form_steps)
        lat = []
        one = ctx.new_result(h, w, 2, u)
        for i in range(12):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.reconstruct(prm, dense=dense[i % nb], out=one)
            b.record()
            b.synchronize()
            if i >= 2:
                lat.append(a.elapsed_time(b))
        # depth error of each point against the nearest true surface of its world pixel
        errs = []
        for o, (_, wd) in zip(outs, made):
            tt = o["t"].cpu().numpy().astype(np.float64)
            al = o["alive"].cpu().numpy().astype(bool)
            truth = wd if u == up else wd[:, 1::up, 1::up]      # pixel grid: the block's centre
            tru = np.where(np.isfinite(truth), truth, np.inf)
            errs.append(np.min(np.abs(tt[:, None] - tru[None]), axis=1)[al])
        e = np.concatenate(errs)
        ok = e < 3.0
        res[name] = {"frames_per_s": round(nb / (ms / 1000), 2),
                     "frame_latency_ms_p50": round(float(np.percentile(lat, 50)), 3),
                     "frame_latency_ms_p99": round(float(np.percentile(lat, 99)), 3),
                     "points_per_frame": int(round(e.size / nb)),
                     "depth_rmse_bins_within_3": round(float(np.sqrt(np.mean(e[ok] ** 2))), 4),
                     "frac_within_3_bins": round(float(ok.mean()), 4)}
    assert ctx.device_status() == R.RT3D_OK
    ctx.close()
    return res


def _pinned(shape, dtype):
    import torch
    return torch.zeros(shape, dtype=dtype).pin_memory().numpy()


def run_e2e(args, ctx, prm, dense, R):
    """The same metric through rt3d_reconstruct_batch_host: every step copies
    the step's frames from page-locked host memory, reconstructs them as one
    batch and copies the results back (also page-locked).  Two input forms of
    the same photons (bitwise-identical results): the dense uint16 histograms
    the benchmark synthesises, and their sparse (offsets, entries) list, the
    form a photon-counting sensor's time tags arrive in."""
    import torch
    nb = len(dense)
    outs = [dict(t=_pinned((K, H, W), torch.float32), r=_pinned((K, H, W), torch.float32),
                 alive=_pinned((K, H, W), torch.uint8), b=_pinned((H, W), torch.float32),
                 n_points=_pinned((1,), torch.int32)) for _ in range(nb)]
    d2h = nb * (K * H * W * 9 + H * W * 4 + 4)
    res = {}
    host_dense = [dict(dense=d.view(torch.int16).cpu().pin_memory().numpy().view(np.uint16)) for d in dense]
    host_csr = []
    for d in dense:
        off, ent = ctx.compact(d)
        o = torch.from_numpy(off.cpu().numpy().astype(np.uint32).view(np.int32)).pin_memory().numpy().view(np.uint32)
        e = torch.from_numpy(ent.cpu().numpy().astype(np.uint32).view(np.int32)).pin_memory().numpy().view(np.uint32)
        host_csr.append(dict(csr=(o, e, (H, W, T))))
    for form, frames in (("dense", host_dense), ("sparse", host_csr)):
        R.reconstruct_batch_host(ctx, prm, frames, outs)          # warm-up (staging, graph)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            R.reconstruct_batch_host(ctx, prm, frames, outs)
        dt = time.perf_counter() - t0
        if form == "dense":
            h2d = nb * H * W * T * 2
            path = "rt3d_reconstruct_batch_host, dense uint16 histograms in page-locked host memory"
        else:
            h2d = sum(f["csr"][0].nbytes + f["csr"][1].nbytes for f in frames)
            path = ("rt3d_reconstruct_batch_host, sparse (offsets, bin<<16|count entries) lists of the same "
                    "photons in page-locked host memory")
        res[form] = {"value": round(nb * args.e2e_steps / dt, 2), "unit": UNIT,
                     "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h, "path": path}
    return res


def oracle_parity(z, irf_samples, irf_origin, prm, out, h, w, t) -> dict:
    """Error of one reconstructed frame (`out`, the library's result tensors)
    against the FP64 oracle on the same histogram `z`.  The oracle's probe
    ensemble (oracle.compare: the oracle's loop with its state rounded after
    every step as FP32 kernels round theirs, at three perturbation sizes)
    marks the points the method itself moves under a perturbation of that
    size; the error is reported over the other points, over all points, and
    on the ill-conditioned ones against the probes' own deviation."""
    import oracle
    from oracle import compare
    irf = oracle.OIrf(irf_samples, irf_origin)
    o, probes = compare.reconstruct_with_probes(z, irf, prm)
    g = {k: v.cpu().numpy() for k, v in out.items() if k != "n_points"}
    st = compare.cloud_stats(g, o, probes, t, 1e-3, 1e-4, r_min=prm["r_min"])
    return {"points": st["points"], "ill_conditioned": st["ill"],
            "alive_mismatch_well_conditioned": st["flips"],
            "dt_max_bins_well_conditioned": st["dt_max"],
            "dt_p999_bins_well_conditioned": st["dt_p999"],
            "dr_max_rel_well_conditioned": st["dr_max"],
            "ill_conditioned_flips": st["ill_flips"],
            "ill_conditioned_flips_no_probe_flips": st["ill_flips_unexplained"],
            "ill_conditioned_over_3x_probe_deviation": st["ill_over_bound"],
            "ill_conditioned_worst_ratio_to_probe": st["ill_ratio_max"],
            "db_max_rel_well_conditioned": st["db_max"],
            "ill_conditioned_backgrounds": st["ill_background_pixels"],
            "ill_backgrounds_over_3x_probe_deviation": st["ill_background_over_bound"],
            "near_threshold_points": st.get("near_threshold", 0),
            "alive_mismatch": st["all_alive_mismatch"],
            "dt_max_bins": st["all_dt_max"], "dt_p999_bins": st["all_dt_p999"],
            "frac_within_1e-3_bins": st["all_frac_within_tol"]}


def _parity_of_frame(oracle, prm, seed, out) -> dict:
    """Parity of the benchmark's frame `seed` (its result `out`) against the oracle."""
    sc = scenes.net_object_wall(H, W, T, seed=seed)
    z = oracle.synthesize(scenes.sampling_tables(sc))
    return oracle_parity(z, sc.irf.samples, sc.irf.origin, prm, out, H, W, T)


def cpu_baseline(args, prm, parity_frame=None):
    """The FP64 oracle, as it stands, on whole frames on this host's cores;
    with parity_frame = (seed, result of the benchmark's first frame), also
    that frame's error against the oracle.  Returns (baseline, parity)."""
    import oracle
    oracle.build()
    zs = []
    for f in range(args.cpu_frames):
        sc = scenes.net_object_wall(H, W, T, seed=1000 + f)
        zs.append((sc, oracle.synthesize(scenes.sampling_tables(sc))))
    irf = oracle.OIrf(zs[0][0].irf.samples, zs[0][0].irf.origin)
    t0 = time.perf_counter()
    for sc, z in zs:
        oracle.reconstruct(z, irf, prm)
    dt = time.perf_counter() - t0
    base = {"value": round(len(zs) / dt, 4), "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{len(zs)} full 141x141x4096 frames (init + 20 iterations), FP64, OpenMP"}
    if args.cpu_single_frames > 0:
        # the same oracle on one host thread
        cores = oracle.num_threads()
        oracle.set_num_threads(1)
        t0 = time.perf_counter()
        for sc, z in zs[:args.cpu_single_frames]:
            oracle.reconstruct(z, irf, prm)
        dt1 = time.perf_counter() - t0
        oracle.set_num_threads(cores)
        base["single_thread"] = {"value": round(args.cpu_single_frames / dt1, 4), "unit": UNIT, "cores": 1,
                                 "sample": f"{args.cpu_single_frames} full 141x141x4096 frame(s), FP64, "
                                           f"one thread"}
    parity = _parity_of_frame(oracle, prm, *parity_frame) if parity_frame is not None else None
    return base, parity


def run_serving(args, device: int, learned_form: bool = False, rate_hz: float = 500.0,
                seconds: float = None) -> dict:
    """Continuous batching of 16 scene streams of mixed frame size (32x32, 64x64,
    141x141, 256x256 pixels; 1024 or 4096 bins), moving 1 bin per frame, with
    Poisson arrivals at 500 frames/s in total; each frame warm-starts from its
    stream's device-resident point cloud.  Each stream cycles through 4
    pre-synthesised frames (device-resident inputs).  learned_form: the
    committed network stands in for APSS (with its fallback)."""
    import torch
    from paper_1905_06700_b300 import rt3d as R
    from paper_1905_06700_b300.serve import GpuBackend, Request, Server, SlotLimits, poisson_arrivals, summarize
    side = [32, 64, 141, 256]
    tbins = [1024, 4096]
    sizes = [(side[s % 4], side[s % 4], tbins[(s // 4) % 2]) for s in range(16)]
    irf = scenes.gamma_irf(3.0, 5.0, 80)
    synth = R.Context(256, 256, 4096, 3, irf.samples, irf.origin, device=device)
    ring = 4
    frames = {}
    for s, (h, w, t) in enumerate(sizes):
        base = scenes.net_object_wall(h, w, t, seed=500 + s, irf=irf)
        for k in range(ring):
            frames[(s, k)] = synth.synthesize(scenes.sampling_tables(scenes.moving_frame(base, k)))
    torch.cuda.synchronize()
    synth.close()
    prm = scenes.make_params(scenes.net_object_wall(64, 64, 4096, irf=irf))
    net = None
    if learned_form:
        from paper_1905_06700_b300 import learned
        if not os.path.exists(WEIGHTS):
            return {"unavailable": "no trained checkpoint"}
        theta, _ = learned.load(WEIGHTS)
        net = R.Net(1, 16, 16, device=device)
        net.set_params(theta)
        prm = dict(prm, depth_denoiser=2)
    lim = SlotLimits(max_frames=16, max_pixels=4 * 256 * 256, max_entries=2 * 256 * 256 * 4096,
                     max_h=256, max_w=256, max_t=4096, mem_budget=4 << 30, k_max=3)
    seconds = args.serve_seconds if seconds is None else seconds
    reqs = poisson_arrivals(16, rate_hz, seconds, sizes, seed=7)
    for r in reqs:
        r.payload = frames[(r.stream, r.index % ring)]
    be = GpuBackend(2, lim, irf.samples, irf.origin, prm, k_max=3, frame_source=None, device=device,
                    depth_net=net)
    warm = [Request(s, 0, *sizes[s], 0.0) for s in range(16)]       # capture the graphs once
    for r in warm:
        r.payload = frames[(r.stream, 0)]
    Server(be).run(warm, timeout_s=120)
    be.state.clear()
    srv = Server(be)
    done = srv.run(reqs, timeout_s=120)
    out = summarize(done)
    out.update({"form": "learned" if learned_form else "plain",
                "offered_frames_per_s": rate_hz, "seconds_offered": seconds, "streams": 16, "slots": 2,
                "batches": len(srv.batches), "mean_batch": len(done) / max(1, len(srv.batches)),
                "device_memory_budget_bytes": lim.mem_budget, "peak_frame_bytes_in_use": srv.peak_bytes,
                "sizes": "32^2, 64^2, 141^2, 256^2 x T 1024/4096, K=3, 20 iterations, warm starts",
                "clock": "host perf_counter, arrival to completion event observed"})
    for c in be.ctx:
        c.close()
    return out


# --------------------------------------------------------------------------- reference arm

def run_reference(args, world, rank):
    """The reference arm is the FP64 oracle on the host cores (no code of the
    paper exists to run): each step reconstructs one full frame."""
    if rank != 0:
        return None
    import oracle
    oracle.build()
    base = scenes.net_object_wall(H, W, T)
    prm = scenes.make_params(base)
    irf = oracle.OIrf(base.irf.samples, base.irf.origin)
    zs = []
    for f in range(args.warmup + args.steps):
        sc = scenes.net_object_wall(H, W, T, seed=1 + f)
        zs.append(oracle.synthesize(scenes.sampling_tables(sc)))
    for f in range(args.warmup):
        oracle.reconstruct(zs[f], irf, prm)
    times = []
    for f in range(args.steps):
        t0 = time.perf_counter()
        oracle.reconstruct(zs[args.warmup + f], irf, prm)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps / total
    cores = oracle.num_threads()
    sample = "1 full 141x141x4096 frame per step (init + 20 iterations), FP64 oracle, OpenMP"
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * total / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(world), "frames_per_step": 1,
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        res = run_reference(args, world, rank)
    else:
        res = run_ours(args, world, rank, local)
    if res is not None and rank == 0:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
