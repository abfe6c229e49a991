#!/usr/bin/env python
"""Benchmark of the stereo visual frontend on GB300: stereo frames/s and p50/p99
per-frame latency.

Workload (plain frontend at sequence scale): a 200-frame 752x480 uint8
stereo sequence of a textured plane under a smooth random camera trajectory
(per-frame motion up to 15 px), 4-level pyramid, a 20x15 grid of 37x32-px
cells with k = 1 (300 keypoints per image), FP32 tracking with the
forward-backward check. One step = one stereo frame through the whole
frontend (pyramid, temporal tracking, detection, stereo matching). Frames are
resident in HBM (144 MB, above the 129 MB L2; each frame is read once per
pass of the sequence).

Reported beside it: end to end through the C ABI from pinned host memory
(upload, step, read-back, one host wait per frame), per-stage times, the
roofline of the dominant kernel, a pyramid+detection HBM roofline pass over a
1.1 GB device-resident batch, and the CPU oracle timed on the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stereo frames/s + p99 frame latency on 1 GB300, plain vs batched+learned-init"
UNIT = "stereo frames/s"
W, H, N_FRAMES, LEVELS = 752, 480, 200, 4
CELL_W, CELL_H, K_CELL, MOTION = 37, 32, 1, 15.0
CAPACITY = 2 * (W // CELL_W) * (H // CELL_H) * K_CELL
WORKLOAD = ("plain frontend: 200-frame 752x480 uint8 stereo sequence, 4-level pyramid, "
            "20x15 cells of 37x32 px, k=1 (300 keypoints/image), FP32 KLT with FB check")
CONFIG = {"workload": WORKLOAD, "frames": N_FRAMES, "w": W, "h": H, "levels": LEVELS,
          "cells": "20x15 of 37x32 px", "k_per_cell": K_CELL, "max_motion_px": MOTION,
          "capacity_per_camera": CAPACITY, "streams": 1,
          "l2": "inputs larger than L2: 144 MB of resident frames, each read once per pass"}

# algorithmic FP32 operations of one keypoint through one direction at one
# level of the KLT: template 52 x ~72 + 5 Gauss-Newton steps of 52 x ~26
FLOPS_PER_KP_DIR_LEVEL = 52 * 72 + 5 * 52 * 26


def seq_seed(rank: int) -> int:
    return 1000 * 2 + rank


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in self.out.strip().splitlines() if r.strip()]
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    i = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[i]


def make_frames(rank: int):
    from paper_2609_30459_gb300 import synth
    seq = synth.make_sequence(seq_seed(rank), N_FRAMES, W, H, 1, max_motion=MOTION)
    return seq.frames                                    # (F, 2, H, W) uint8


def oracle_frames_per_s(frames, n_frames, warmup=2):
    """The CPU oracle frontend, as it stands, over a bounded sample of frames."""
    import oracle
    from oracle import frontend as ofe
    oracle.build()
    cores = os.cpu_count() or 1
    p = ofe.Params(n_levels=LEVELS, cell_w=CELL_W, cell_h=CELL_H, k=K_CELL)
    st = ofe.StreamState()
    for f in range(warmup):
        ofe.step(st, frames[f % N_FRAMES], p, CAPACITY, n_threads=cores)
    times = []
    for f in range(warmup, warmup + n_frames):
        t0 = time.perf_counter()
        ofe.step(st, frames[f % N_FRAMES], p, CAPACITY, n_threads=cores)
        times.append(time.perf_counter() - t0)
    return len(times) / sum(times), cores, times


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    frames = make_frames(0)
    fps, cores, times = oracle_frames_per_s(frames, args.steps, args.warmup)
    sample = (f"{args.steps} consecutive frames (after {args.warmup} warm-up frames) of the "
              f"200-frame sequence through the FP64 oracle frontend, tracking threaded over "
              f"{cores} cores")
    line = {"metric": METRIC, "value": fps, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": CONFIG, "impl": "reference",
            "p50_ms": 1000 * percentile(times, 50), "p99_ms": 1000 * percentile(times, 99),
            "cpu_baseline": {"value": fps, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": fps, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def pyramid_detect_roofline(torch, vio, frames_dev, peaks, peak_src):
    """Pyramid and detection of a device-resident batch well above L2 (the 400
    images of the sequence, repeated to ~1.1 GB): vio_pyramid_detect, one fused
    launch plus the selection launch, timed with CUDA events."""
    reps = 8
    imgs = frames_dev.reshape(-1, H, W).repeat(reps, 1, 1).contiguous()   # (3200, H, W)
    n = imgs.shape[0]
    params = vio.default_params(n_levels=LEVELS, cell_w=CELL_W, cell_h=CELL_H,
                                k_per_cell=K_CELL)
    ctx = vio.Context(params, W, H, n)
    pyr = vio.Pyramids(imgs, LEVELS)
    gx, gy = W // CELL_W, H // CELL_H
    cap = gx * gy * K_CELL
    kp = torch.empty((n, cap, 2), dtype=torch.float32, device=imgs.device)
    sc = torch.empty((n, cap), dtype=torch.int16, device=imgs.device)
    cnt = torch.empty(n, dtype=torch.int32, device=imgs.device)
    s = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    times = []
    for it in range(6):
        ev[0].record(s)
        ctx.pyramid_detect(pyr, kp, sc, cnt, cap)
        ev[1].record(s)
        torch.cuda.synchronize()
        if it >= 2:
            times.append(ev[0].elapsed_time(ev[1]) / 1000)
    L = pyr.layout
    upper = sum(L.w[l] * L.h[l] for l in range(1, LEVELS))
    n_kp = int(cnt.sum().item())
    alg = n * (W * H + upper) + n_kp * 10
    t = statistics.median(times)
    gbs = alg / t / 1e9
    ctx.close()
    return {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / peaks["hbm_gbs"], "traffic": None, "kernel": "frame_front_kernel",
            "images": n, "batch_bytes_in": n * W * H, "algorithmic_bytes": alg,
            "algorithmic_bytes_per_image": W * H + upper + n_kp * 10 / n,
            "ms": 1000 * t, "peak_source": peak_src,
            "note": "vio_pyramid_detect: pyramid levels 1-3 and per-cell FAST/NMS/top-k in one "
                    "launch, then the per-image selection; level 0 read once, upper levels "
                    "and 10 B per keypoint written"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-frames", type=int, default=60)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2609_30459_gb300 import vio
    vio.load(build=True)
    peaks, peak_src = load_peaks()

    frames_np = make_frames(rank)
    frames = torch.from_numpy(frames_np).cuda()                 # (F, 2, H, W) resident
    params = vio.default_params(n_levels=LEVELS, cell_w=CELL_W, cell_h=CELL_H,
                                k_per_cell=K_CELL)
    fe = vio.Frontend(params, W, H, 1, CAPACITY)
    stream = torch.cuda.current_stream()

    # warm-up on the last frames of the sequence, then a fresh start at frame 0
    for i in range(args.warmup):
        fe.step(frames[N_FRAMES - args.warmup + i: N_FRAMES - args.warmup + i + 1])
    torch.cuda.synchronize()
    fe.reset()
    fe.set_timing(True)
    _, steps_before = fe.read_stats()

    frames5 = frames.view(N_FRAMES, 1, 2, H, W)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        time.sleep(0.5)                        # let the sampler start before timing
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        torch.cuda.nvtx.range_push("timed")
        ev0.record(stream)
        left = args.steps
        while left > 0:                        # whole passes of the sequence, one call each
            n = min(N_FRAMES, left)
            fe.run(frames5[:n])
            left -= n
        ev1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if world > 1:
            dist.barrier()
    total_s = ev0.elapsed_time(ev1) / 1000.0
    stage_ms, n_timed, step_ms = fe.read_timing(max_steps=args.steps)
    fe.set_timing(False)
    stats, steps_after = fe.read_stats()
    idx = [(steps_before + k) % vio.STATS_RING for k in range(args.steps)]
    st = stats[idx, 0, :].astype(np.int64)                       # (K, 7)
    tracked = int(st[:, 0].sum() + st[:, 1].sum())
    new_kp = int(st[:, 4].sum())
    stereo_in = int(st[:, 6].sum())                               # candidates matched
    survived = int(st[:, 2].sum() + st[:, 3].sum())

    t_max = total_s
    if world > 1:
        tt = torch.tensor([total_s], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    value = world * args.steps / t_max

    # dominant kernel: the stage with the largest share of the step
    per_stage = {k: v / max(n_timed, 1) for k, v in stage_ms.items()}
    dom = max(per_stage, key=per_stage.get)
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12               # TFLOP/s
    if dom == "track":     # temporal tracks and stereo candidates, both with FB
        flops = (tracked + stereo_in) * 2 * LEVELS * FLOPS_PER_KP_DIR_LEVEL
        t_launch = stage_ms["track"] / 1000.0
    else:
        flops, t_launch = None, None
    roofline = None
    if flops is not None and t_launch:
        ach = flops / t_launch / 1e12
        roofline = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": ach / fp32_peak, "traffic": None, "kernel": "frame_track_kernel",
                    "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock "
                                   f"{sm_max:.0f} MHz ({peak_src} clock)",
                    "avg_launch_us": 1e6 * t_launch / args.steps}

    # end to end through the C ABI from pinned host memory, one wait per frame
    e2e = None
    if rank == 0 or world > 1:
        host = torch.from_numpy(frames_np).pin_memory()
        slots = torch.empty((2, 1, 2, H, W), dtype=torch.uint8, device="cuda")
        out_xy = torch.empty((1, 2, CAPACITY, 2), dtype=torch.float32).pin_memory()
        out_id = torch.empty((1, 2, CAPACITY), dtype=torch.int32).pin_memory()
        out_cnt = torch.empty((1, 2), dtype=torch.int32).pin_memory()
        out_new = torch.empty((1, CAPACITY, 2), dtype=torch.float32).pin_memory()
        out_nc = torch.empty((1,), dtype=torch.int32).pin_memory()
        fe.reset()
        v = fe.view()
        lat = []

        def one(k):
            f = k % N_FRAMES
            slot = slots[k % 2]
            slot.copy_(host[f: f + 1], non_blocking=True)
            fe.step(slot)
            vv = fe.view()
            out_xy.copy_(vv["track_xy"], non_blocking=True)
            out_id.copy_(vv["track_id"], non_blocking=True)
            out_cnt.copy_(vv["track_count"], non_blocking=True)
            out_new.copy_(vv["new_xy"], non_blocking=True)
            out_nc.copy_(vv["new_count"], non_blocking=True)
            stream.synchronize()

        for k in range(args.warmup):
            one(N_FRAMES - args.warmup + k)
        fe.reset()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            ts = time.perf_counter()
            one(k)
            lat.append(time.perf_counter() - ts)
        e2e_s = time.perf_counter() - t0
        if world > 1:
            tt = torch.tensor([e2e_s], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e2e_s = float(tt.item())
        del v
        bo = sum(t.numel() * t.element_size() for t in (out_xy, out_id, out_cnt, out_new,
                                                          out_nc))
        e2e = {"value": world * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 2 * H * W, "d2h_bytes_per_step": bo,
               "p50_ms": 1000 * percentile(lat, 50), "p99_ms": 1000 * percentile(lat, 99)}

    pd = pyramid_detect_roofline(torch, vio, frames, peaks, peak_src) if rank == 0 else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fps, cores, _ = oracle_frames_per_s(frames_np, args.cpu_frames)
        cpu = {"value": fps, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_frames} consecutive frames of the same sequence through the "
                         f"FP64 oracle frontend (after 2 warm-up frames), tracking threaded "
                         f"over {cores} cores"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8+f32", "data": "synthetic", "config": CONFIG,
            "p50_ms": percentile(step_ms, 50), "p99_ms": percentile(step_ms, 99),
            "tracked_keypoints_per_s": world * tracked / t_max,
            "stage_ms_per_step": per_stage,
            "keypoints_per_step": {"temporal": tracked / args.steps,
                                   "survived": survived / args.steps,
                                   "new": new_kp / args.steps,
                                   "stereo_candidates": stereo_in / args.steps},
            "gpu_launches": args.steps * fe.launches_per_step(),
            "e2e": e2e, "roofline": roofline, "pyramid_detect_roofline": pd,
            "cpu_baseline": cpu, "clocks": clk.summary(),
            "host_wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    fe.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
