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
(upload, step, read-back; pipelined, and with one host wait per frame), the
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
# ncu counters of frame_track_kernel on this workload (the profile summary in
# profiles/ names the command)
TRACK_NCU = {"profile": "profiles/frame_kernels_752x480.md"}
# DRAM bytes (read + write) per image of the pyramid+detection pass
# (vio_pyramid_detect: pyr_pass_kernel, detect_cells_kernel, select_kernel),
# from an ncu capture of 512 images of the headline sequence with the L2 kept
# between launches (profiles/pyramid_detect_752x480x512.md names the command);
# a full launch moves this per image
PYRDET_TRAFFIC_PER_IMAGE = 808243


def seq_seed(rank: int) -> int:
    """Each rank runs its own sequence (weak scaling: streams are independent)."""
    return 1000 * 2 + rank


def max_over_ranks(value: float, dist=None, device: str = "cpu") -> float:
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def _find_number(d, key):
    """The first numeric value stored under `key` in a (possibly nested) dict."""
    if isinstance(d, dict):
        v = d.get(key)
        if isinstance(v, (int, float)) and not isinstance(v, bool) and v > 0:
            return float(v)
        for x in d.values():
            r = _find_number(x, key)
            if r is not None:
                return r
    return None


def section(name, fn):
    """fn() for one optional part of the report; an exception there is
    reported as {"error": ...} in its place (traceback on stderr), so the
    headline line is still printed."""
    import traceback
    try:
        return fn()
    except Exception as e:                       # noqa: BLE001 - reported, not hidden
        traceback.print_exc()
        return {"error": f"{name}: {type(e).__name__}: {e}"[:500]}


def load_peaks(path=None):
    """The measured HBM copy bandwidth and BF16 GEMM rate of this machine's GPUs
    (MEASURED_PEAKS.json, flat or nested), else the fallback figures; each
    missing figure falls back on its own, and the source says which."""
    path = path or os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS), "fallback"
    out, missing = {}, []
    for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained"):
        v = _find_number(d, k)
        if v is not None:
            out[k] = v
        elif k in FALLBACK_PEAKS:
            out[k] = FALLBACK_PEAKS[k]
            missing.append(k)
    if "hbm_gbs" in missing and "bf16_tflops" in missing:
        return dict(FALLBACK_PEAKS), "fallback"
    return out, "measured" if not missing else "measured (fallback: " + ", ".join(missing) + ")"


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


def oracle_frames_per_s(frames, n_frames, warmup=2, cores=None, budget_s=None):
    """The CPU oracle frontend, as it stands, over a bounded sample of frames
    (tracking threaded over `cores` host cores, all of them by default); with
    budget_s, the timed frames stop once they have taken that long."""
    import oracle
    from oracle import frontend as ofe
    oracle.build()
    cores = cores or os.cpu_count() or 1
    p = ofe.Params(n_levels=LEVELS, cell_w=CELL_W, cell_h=CELL_H, k=K_CELL)
    st = ofe.StreamState()
    for f in range(warmup):
        ofe.step(st, frames[f % N_FRAMES], p, CAPACITY, n_threads=cores)
    times = []
    for f in range(warmup, warmup + n_frames):
        t0 = time.perf_counter()
        ofe.step(st, frames[f % N_FRAMES], p, CAPACITY, n_threads=cores)
        times.append(time.perf_counter() - t0)
        if budget_s is not None and sum(times) >= budget_s:
            break
    return len(times) / sum(times), cores, times


def accuracy_vs_oracle(torch, vio, frames, levels, cw, ch, k, n_frames, params_kw=None):
    """Flow error and track-status agreement of the GPU frontend against the
    FP64 oracle frontend, step by step on the first n_frames of `frames`
    ((F, 2 * streams, h, w) uint8): before each frame the oracle receives the
    GPU's lists, so each step is compared on the same inputs. Per step and
    stream: every temporal track and every stereo match of a new keypoint is
    compared by id (position error where both keep it; agreement = both keep
    it or both drop it); new detections are compared bit for bit."""
    import numpy as np
    import oracle
    from oracle import frontend as ofe
    oracle.build()
    params_kw = dict(params_kw or {})
    F, C, h, w = frames.shape
    ns = C // 2
    p = vio.default_params(n_levels=levels, cell_w=cw, cell_h=ch, k_per_cell=k, **params_kw)
    op = ofe.Params(n_levels=levels, cell_w=cw, cell_h=ch, k=k,
                    thresholds=tuple(params_kw.get("thresholds", (40, 20, 10, 5))),
                    gn_iters=params_kw.get("gn_iters", 5))
    cap = 2 * (w // cw) * (h // ch) * k
    fe = vio.Frontend(p, w, h, ns, cap)
    dev = torch.from_numpy(np.ascontiguousarray(frames[:n_frames])).cuda().view(
        n_frames, ns, 2, h, w)
    states = [ofe.StreamState() for _ in range(ns)]
    errs, agree, n_cmp, new_same, new_total = [], 0, 0, 0, 0
    for t in range(n_frames):
        fe.step(dev[t])
        torch.cuda.synchronize()
        v = fe.view()
        for s in range(ns):
            st = states[s]
            prev_ids = [st.ids[0].copy(), st.ids[1].copy()]
            ofe.step(st, frames[t, 2 * s: 2 * s + 2], op, cap, n_threads=os.cpu_count() or 1)
            cnt = v["track_count"][s].cpu().numpy()
            gxy = [v["track_xy"][s, c, : cnt[c]].cpu().numpy() for c in range(2)]
            gid = [v["track_id"][s, c, : cnt[c]].cpu().numpy() for c in range(2)]
            g_new = int(v["new_count"][s])
            for c in range(2):
                gpos = dict(zip(gid[c].tolist(), gxy[c].astype(np.float64)))
                opos = dict(zip(st.ids[c].tolist(), st.xy[c].astype(np.float64)))
                judged = set(prev_ids[c].tolist())
                if c == 1:                       # this step's stereo matches too
                    judged |= set(gid[0][len(gid[0]) - g_new:].tolist())
                for i in judged:
                    n_cmp += 1
                    agree += (i in gpos) == (i in opos)
                    if i in gpos and i in opos:
                        errs.append(float(np.abs(gpos[i] - opos[i]).max()))
            # detections: the oracle's, given the GPU's camera-0 survivors
            g_new_xy = v["new_xy"][s, :g_new].cpu().numpy()
            occ = ofe.occupancy(gxy[0][: max(int(cnt[0]) - g_new, 0)], w, h, cw, ch)
            o_new_xy, _ = oracle.detect_grid(frames[t, 2 * s], cw, ch, k=k,
                                             thresholds=op.thresholds, border=p.detect_border,
                                             occupancy=occ)
            new_total += 1
            new_same += int(np.array_equal(g_new_xy, o_new_xy))
            # the next step starts from the GPU's lists
            st.xy = [gxy[0].copy(), gxy[1].copy()]
            st.ids = [gid[0].copy(), gid[1].copy()]
    fe.close()
    e = np.array(errs) if errs else np.zeros(1)
    return {"frames": n_frames, "streams": ns, "compared_tracks": n_cmp,
            "max_flow_err_px": float(e.max()), "p99_flow_err_px": float(np.percentile(e, 99)),
            "status_agree": agree / max(n_cmp, 1),
            "detections_bit_exact": new_same / max(new_total, 1)}


def accuracy_report(torch, vio, frames_np):
    """Flow error and status agreement against the FP64 oracle for cfg 1, 2
    and 3 and the lite parameters (accuracy_vs_oracle on a few frames each)."""
    import numpy as np
    from paper_2609_30459_gb300 import synth
    out = {}
    d = synth.stereo_pair_small_motion(1001, W, H)               # cfg 1: t and t + 1
    out["cfg1"] = accuracy_vs_oracle(torch, vio, d["images"], 3, 94, 60, 2, 2)
    out["cfg2"] = accuracy_vs_oracle(torch, vio, frames_np, LEVELS, CELL_W, CELL_H, K_CELL, 12)
    seqs = [synth.make_sequence(3000 + i, 4, 1920, 1080, 1, max_motion=40.0,
                                tex_size=2048).frames for i in range(2)]
    out["cfg3"] = accuracy_vs_oracle(torch, vio, np.concatenate(seqs, 1), 5, 48, 43, 1, 4)
    out["lite"] = accuracy_vs_oracle(torch, vio, frames_np, LEVELS, 82, 82, 1, 12,
                                     params_kw={"gn_iters": 3, "thresholds": (40, 20)})
    out["note"] = ("GPU frontend vs the FP64 oracle frontend, step by step with the GPU's lists "
                   "handed to the oracle before each frame; flow error in level-0 px over the "
                   "tracks both keep; status_agree over every temporal track and stereo match; "
                   "cfg3 = the same seeds as other_configs[0]")
    return out


# the reference arm's timed frames end after this long, whatever the step count
REFERENCE_BUDGET_S = 150.0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    frames = make_frames(0)
    fps, cores, times = oracle_frames_per_s(frames, args.steps, args.warmup,
                                            budget_s=REFERENCE_BUDGET_S)
    capped = (f" (the first {len(times)} of the {args.steps} requested: the timed frames stop "
              f"after {REFERENCE_BUDGET_S:.0f} s)" if len(times) < args.steps else "")
    sample = (f"{len(times)} consecutive frames{capped}, after {args.warmup} warm-up frames, of "
              f"the 200-frame sequence through the FP64 oracle frontend, tracking threaded over "
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


def pyramid_detect_roofline(torch, vio, frames_dev, peaks, peak_src, w=None, h=None,
                            levels=None, cw=None, ch=None, reps=8):
    """Pyramid and detection of a device-resident batch well above L2 (the
    headline's 400 images repeated to ~1.1 GB, or cfg 3's 400 images of
    1920x1080): vio_pyramid_detect, one fused launch plus the selection launch,
    timed with CUDA events."""
    w, h = w or W, h or H
    levels, cw, ch = levels or LEVELS, cw or CELL_W, ch or CELL_H
    imgs = frames_dev.reshape(-1, h, w)
    if reps > 1:
        imgs = imgs.repeat(reps, 1, 1)
    imgs = imgs.contiguous()
    n = imgs.shape[0]
    params = vio.default_params(n_levels=levels, cell_w=cw, cell_h=ch, k_per_cell=K_CELL)
    ctx = vio.Context(params, w, h, n)
    pyr = vio.Pyramids(imgs, levels)
    gx, gy = w // cw, h // ch
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
    upper = sum(L.w[l] * L.h[l] for l in range(1, levels))
    n_kp = int(cnt.sum().item())
    alg = n * (w * h + upper) + n_kp * 10
    t = statistics.median(times)
    gbs = alg / t / 1e9
    ctx.close()
    traffic = None
    if PYRDET_TRAFFIC_PER_IMAGE and (w, h, levels, cw, ch) == (W, H, LEVELS, CELL_W, CELL_H):
        traffic = PYRDET_TRAFFIC_PER_IMAGE * n
    return {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / peaks["hbm_gbs"], "traffic": traffic,
            "traffic_note": "DRAM read + write bytes per launch: an ncu capture of 512 images (L2 kept "
                            "between launches) "
                            "scaled by the images of this launch",
            "kernel": "vio_pyramid_detect (pyr_pass_kernel, detect_cells_kernel, select_kernel)",
            "images": n, "image": f"{w}x{h}, {levels} levels, {gx}x{gy} cells",
            "batch_bytes_in": n * w * h, "algorithmic_bytes": alg,
            "algorithmic_bytes_per_image": w * h + upper + n_kp * 10 / n,
            "ms": 1000 * t, "peak_source": peak_src,
            "note": "vio_pyramid_detect: per chunk of images (level 0 at most 64 MiB) the "
                    "pyramid launch (levels 1-2, then 3) and the per-cell FAST/NMS/top-k "
                    "launch, then the per-image selection; algorithmic bytes: level 0 read "
                    "once, upper levels and 10 B per keypoint written"}


def selection_variants(torch, vio, frames_dev, w, h, levels, cw, ch, reps=5):
    """The paper's per-cell selections (Sec. III-D) timed on one device-resident
    batch through vio_pyramid_detect: k rounds of a warp maximum, a bitonic
    k-sort and (k = 1) an atomic maximum, for k = 1 and k = 4; every mode must
    give the same keypoints bit for bit."""
    imgs = frames_dev.reshape(-1, h, w).contiguous()
    n = imgs.shape[0]
    pyr = vio.Pyramids(imgs, levels)
    gx, gy = w // cw, h // ch
    out = {"images": n, "image": f"{w}x{h}, {levels} levels, {gx}x{gy} cells of {cw}x{ch} px",
           "ms": {}}
    s = torch.cuda.current_stream()
    for k, modes in ((1, (0, 1, 2)), (4, (0, 1))):
        ref = None
        for mode in modes:
            p = vio.default_params(n_levels=levels, cell_w=cw, cell_h=ch, k_per_cell=k,
                                   select_mode=mode)
            ctx = vio.Context(p, w, h, n)
            cap = gx * gy * k
            kp = torch.zeros((n, cap, 2), dtype=torch.float32, device=imgs.device)
            sc = torch.zeros((n, cap), dtype=torch.int16, device=imgs.device)
            cnt = torch.zeros(n, dtype=torch.int32, device=imgs.device)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            times = []
            for it in range(reps + 2):
                ev[0].record(s)
                ctx.pyramid_detect(pyr, kp, sc, cnt, cap)
                ev[1].record(s)
                torch.cuda.synchronize()
                if it >= 2:
                    times.append(ev[0].elapsed_time(ev[1]))
            res = (cnt.clone(), kp.clone(), sc.clone())
            if ref is None:
                ref = res
            same = all(torch.equal(x, y) for x, y in zip(ref, res))
            name = {0: "warp_max", 1: "bitonic", 2: "atomic_max"}[mode]
            out["ms"][f"k{k}_{name}"] = statistics.median(times)
            out.setdefault("identical", {})[f"k{k}_{name}"] = bool(same)
            ctx.close()
    return out


def model_based_start(torch, vio, seeds=(8200, 8201, 8202), w=640, h=480, levels=5, cell=32,
                      motion=40.0, n_frames=6, f=500.0):
    """The paper's start of a track (Sec. III-E), fed with the generator's
    ground-truth poses in place of a backend prediction: vio_predict_warp, then
    the unchanged pyramidal tracker with the FB check, against the identity
    start. Per frame pair of sequences with up to 40 px of motion: tracks that
    end OK and within 0.5 px of the ground truth."""
    import numpy as np
    from paper_2609_30459_gb300 import synth
    L = levels
    tot = {"identity": 0, "model": 0, "n": 0}
    t_pred = []
    for seed in seeds:
        seq = synth.make_sequence(seed, n_frames, w, h, 1, max_motion=motion, tex_size=2048)
        frames = torch.from_numpy(np.ascontiguousarray(seq.frames[:, 0])).cuda()
        p = vio.default_params(n_levels=L, cell_w=cell, cell_h=cell)
        ctx = vio.Context(p, w, h, n_frames)
        pyr = vio.Pyramids(frames, L)
        cap = (w // cell) * (h // cell)
        kp = torch.empty((n_frames, cap, 2), device="cuda")
        sc = torch.empty((n_frames, cap), dtype=torch.int16, device="cuda")
        cnt = torch.empty(n_frames, dtype=torch.int32, device="cuda")
        ctx.pyramid_detect(pyr, kp, sc, cnt, cap)
        poses, rhos = [], []
        c_img = ((w - 1) / 2.0, (h - 1) / 2.0)
        for t in range(n_frames - 1):
            pa, pb = seq.poses[t][0], seq.poses[t + 1][0]
            # the similarity poses of the generator as pinhole cameras looking
            # at the plane fronto-parallel from depth f * s, rolled by th
            def rz(a):
                return np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
            Ca = np.array([pa.tx, pa.ty, -f * pa.s])
            Cb = np.array([pb.tx, pb.ty, -f * pb.s])
            R = rz(pb.th).T @ rz(pa.th)
            tt = rz(pb.th).T @ (Ca - Cb)
            poses.append(np.concatenate([R.reshape(-1), tt]))
            rhos.append(1.0 / (f * pa.s))
        n = n_frames - 1
        pose = torch.from_numpy(np.array(poses, np.float32)).cuda()
        rho = torch.from_numpy(np.repeat(np.array(rhos, np.float32)[:, None], cap, 1)).cuda()
        pts = kp[:n].contiguous()
        c = cnt[:n].contiguous()
        init = torch.empty((n, cap, 3), device="cuda")
        K = (f, f, c_img[0], c_img[1])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        vio.predict_warp(K, K, pose, pts, rho, c, cap, n, init)
        e1.record()
        out = {}
        for name, ini in (("identity", None), ("model", init)):
            o = torch.empty((n, cap, 3), device="cuda")
            st = torch.empty((n, cap), dtype=torch.uint8, device="cuda")
            ctx.track_patches(pyr, pyr.batch(0, 1, n), pyr.batch(1, 1, n), pts, c, cap, o, st,
                              init=ini)
            out[name] = (o.cpu().numpy(), st.cpu().numpy())
        torch.cuda.synchronize()
        t_pred.append(e0.elapsed_time(e1))
        kph, ch_ = pts.cpu().numpy(), c.cpu().numpy()
        for t in range(n):
            m = int(ch_[t])
            gt = synth.PlanarScene.map_points(seq.poses[t][0], seq.poses[t + 1][0], kph[t, :m],
                                              w, h, seq.c_tex)
            tot["n"] += m
            for name in ("identity", "model"):
                o, st = out[name]
                ok = (st[t, :m] == 0) & (np.abs(o[t, :m, :2] - gt).max(1) < 0.5)
                tot[name] += int(ok.sum())
        ctx.close()
    return {"keypoints": tot["n"],
            "ok_within_0.5px": {k: tot[k] / max(tot["n"], 1) for k in ("identity", "model")},
            "predict_ms_per_launch": statistics.median(t_pred),
            "workload": f"{len(seeds)} sequences of {n_frames} frames, {w}x{h}, motion up to "
                        f"{motion:.0f} px, {levels} levels, {cell}-px cells; poses from the "
                        "generator (pinhole f = 500 px over the textured plane)"}


def lite_vs_standard(torch, vio, seeds=(2000, 2001, 2002), n_frames=12, w=752, h=480,
                     levels=4, motion=15.0):
    """The speed/accuracy trade of the lite parameters (Sec. IV-D: minimum
    FAST threshold 20, 82-px cells, 3 Gauss-Newton iterations) against the
    standard ones (thresholds down to 5, the headline's 37x32-px cells, 5
    iterations) on the same sequences, scored against the generator's ground
    truth: the camera-0 keypoints of frame t tracked (with the FB check) to
    frame t + 1. Per setting: keypoints per frame, the fraction of tracks that
    end OK, the fraction of OK tracks within 0.5 px of the true position, the
    median and p99 error of OK tracks, and the median time of one detection
    and one tracking launch over the n_frames - 1 frame pairs."""
    import numpy as np
    from paper_2609_30459_gb300 import synth
    settings = {"standard": dict(cell_w=CELL_W, cell_h=CELL_H),
                "lite": dict(cell_w=82, cell_h=82, gn_iters=3, thresholds=(40, 20))}
    acc = {k: {"kp": 0, "ok": 0, "true": 0, "err": [], "t_det": [], "t_track": []}
           for k in settings}
    n = n_frames - 1
    for seed in seeds:
        seq = synth.make_sequence(seed, n_frames, w, h, 1, max_motion=motion, tex_size=2048)
        frames = torch.from_numpy(np.ascontiguousarray(seq.frames[:, 0])).cuda()
        for name, kw in settings.items():
            p = vio.default_params(n_levels=levels, **kw)
            cap = (w // p.cell_w) * (h // p.cell_h) * p.k_per_cell
            ctx = vio.Context(p, w, h, n_frames)
            pyr = vio.Pyramids(frames, levels)
            kp = torch.empty((n_frames, cap, 2), device="cuda")
            sc = torch.empty((n_frames, cap), dtype=torch.int16, device="cuda")
            cnt = torch.empty(n_frames, dtype=torch.int32, device="cuda")
            o = torch.empty((n, cap, 3), device="cuda")
            st = torch.empty((n, cap), dtype=torch.uint8, device="cuda")
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            for rep in range(4):                  # the first repetition warms up
                ev[0].record()
                ctx.pyramid_detect(pyr, kp, sc, cnt, cap)
                ev[1].record()
                pts, c = kp[:n].contiguous(), cnt[:n].contiguous()
                ctx.track_patches(pyr, pyr.batch(0, 1, n), pyr.batch(1, 1, n), pts, c, cap, o,
                                  st)
                ev[2].record()
                torch.cuda.synchronize()
                if rep:
                    acc[name]["t_det"].append(ev[0].elapsed_time(ev[1]))
                    acc[name]["t_track"].append(ev[1].elapsed_time(ev[2]))
            kph, ch_, oh, sth = pts.cpu().numpy(), c.cpu().numpy(), o.cpu().numpy(), st.cpu().numpy()
            a = acc[name]
            for t in range(n):
                m = int(ch_[t])
                gt = synth.PlanarScene.map_points(seq.poses[t][0], seq.poses[t + 1][0],
                                                  kph[t, :m], w, h, seq.c_tex)
                ok = sth[t, :m] == 0
                err = np.abs(oh[t, :m, :2] - gt).max(1)[ok]
                a["kp"] += m
                a["ok"] += int(ok.sum())
                a["true"] += int((err < 0.5).sum())
                a["err"].extend(err.tolist())
            ctx.close()
    out = {}
    for name, a in acc.items():
        out[name] = {"keypoints_per_frame": a["kp"] / (n * len(seeds)),
                     "ok": a["ok"] / max(a["kp"], 1),
                     "ok_within_0.5px": a["true"] / max(a["ok"], 1),
                     "median_err_px": percentile(a["err"], 50),
                     "p99_err_px": percentile(a["err"], 99),
                     "detect_ms_per_launch": statistics.median(a["t_det"]),
                     "track_ms_per_launch": statistics.median(a["t_track"])}
    out["workload"] = (f"{len(seeds)} sequences of {n_frames} frames, {w}x{h}, motion up to "
                       f"{motion:.0f} px, {levels} levels; one detection launch over the "
                       f"{n_frames} camera-0 frames, one tracking launch over the {n} pairs; "
                       "error = max-norm distance to the generator's mapped point")
    return out


# Batched + learned initializer: 16 streams, 4 each of these sizes, cells for
# 300 / 300 / 600 / 1000 keypoints per image, 5 levels, motion up to 40 px
CFG4_CLASSES = [(640, 480, 32, 32), (752, 480, 37, 32), (1280, 720, 42, 36), (1920, 1080, 48, 43)]
CFG4_STREAMS, CFG4_FRAMES, CFG4_LEVELS, CFG4_MOTION = 4, 24, 5, 40.0


def _render_cfg4(job):
    from paper_2609_30459_gb300 import synth
    seed, w, h = job
    return synth.make_sequence(seed, CFG4_FRAMES, w, h, 1, max_motion=CFG4_MOTION,
                               tex_size=2048).frames


def cfg4_frames():
    """Per class, per stream: (F, 2, h, w) uint8 frames (seed 4000 + stream),
    rendered by a spawned pool of host processes."""
    import multiprocessing as mp
    jobs = [(4000 + k * CFG4_STREAMS + i, w, h)
            for k, (w, h, _, _) in enumerate(CFG4_CLASSES) for i in range(CFG4_STREAMS)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        out = pool.map(_render_cfg4, jobs)
    return [out[k * CFG4_STREAMS:(k + 1) * CFG4_STREAMS] for k in range(len(CFG4_CLASSES))]


# useful FLOPs of one forward pass of the flow network: three 3x3 stride-2
# convolutions (4 -> 32 channels at 8x8, 32 -> 32 at 4x4 and at 2x2) and the
# dense layers 128 -> 64 -> 3
INITNET_FLOP = (2 * 8 * 8 * 32 * 4 * 9 + 2 * 4 * 4 * 32 * 32 * 9 + 2 * 2 * 2 * 32 * 32 * 9
                + 2 * 128 * 64 + 2 * 64 * 3)


def initnet_tensor_roofline(torch, vio, net, peaks, n=1 << 16, reps=5, peak_src="measured"):
    """The flow network's forward pass on the tcgen05 tensor cores (BF16
    operands, FP32 accumulators in tensor memory) over n random inputs, useful
    FLOPs against the measured dense BF16 peak."""
    g = torch.Generator(device="cuda").manual_seed(11)
    x = (0.5 * torch.randn((n, 4, 16, 16), device="cuda", generator=g)).to(torch.bfloat16)
    x = x.view(torch.int16)
    out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    for _ in range(2):
        net.forward(x, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        net.forward(x, out)
    e1.record(s)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1000.0 / reps
    ach = n * INITNET_FLOP / t / 1e12
    peak = peaks.get("bf16_tflops", 1900.0)
    return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "kernel": "forward_tc_kernel", "samples": n,
            "flop_per_sample": INITNET_FLOP, "ms": 1000 * t,
            "peak_source": f"{peak_src} dense BF16 (burst)",
            "note": "tcgen05.mma (M = 128 rows, operands in shared memory, accumulators in "
                    "tensor memory), rounds of 32 samples per 128-thread CTA; the proposal "
                    "launch of the frame step runs the same code"}


def frontend_config_run(torch, vio, name, w, h, n_streams, levels, cw, ch, n_frames, motion,
                        seed0, steps, params_kw=None, roofline=None):
    """One frontend configuration over its own synthetic sequences (each
    stream its own seed), autotuned launch shapes, device-resident frames
    played forward and back: stereo frames/s (n_streams frames per step) and
    per-step latency from a separate pass that records each step's first and
    last event only."""
    import numpy as np
    from paper_2609_30459_gb300 import synth
    seqs = [synth.make_sequence(seed0 + i, n_frames, w, h, 1, max_motion=motion,
                                tex_size=2048).frames for i in range(n_streams)]
    frames = torch.from_numpy(np.stack(seqs, 1)).cuda()      # (F, streams, 2, h, w)
    order = list(range(n_frames)) + list(range(n_frames - 2, 0, -1))
    p = vio.default_params(n_levels=levels, cell_w=cw, cell_h=ch, **(params_kw or {}))
    cap = 2 * (w // cw) * (h // ch) * p.k_per_cell
    fe = vio.Frontend(p, w, h, n_streams, cap)
    tune, _ = tune_frontend(torch, fe, frames, [(k2, 0, first, k1) for k2 in (32, 64, 128, 256)
                                                for first in (0, 2) for k1 in (128, 256)])
    for t in range(3):
        fe.step(frames[order[t]])
    torch.cuda.synchronize()
    _, steps0 = fe.read_stats()
    # the timed steps in one native call over the frames in play order (no
    # per-step host work between them)
    play = frames[torch.tensor([order[(t + 3) % len(order)] for t in range(steps)],
                               device=frames.device)]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fe.run(play)
    e1.record()
    torch.cuda.synchronize()
    total_s = e0.elapsed_time(e1) / 1000.0
    stats, _ = fe.read_stats()
    idx = [(steps0 + k) % vio.STATS_RING for k in range(steps)]
    st = stats[idx].astype(np.int64)
    fe.set_timing(2)              # each step's first and last event only
    fe.reset()
    for t in range(min(steps, 200)):
        fe.step(frames[order[t % len(order)]])
    _, n_t, step_ms = fe.read_timing(max_steps=200)
    fe.close()
    pd = None
    if roofline is not None:       # all frames of all cameras as one detection batch
        pd = pyramid_detect_roofline(torch, vio, frames, *roofline, w=w, h=h, levels=levels,
                                     cw=cw, ch=ch, reps=1)
    return {"config": name, "pyramid_detect_roofline": pd, "w": w, "h": h, "stereo_streams": n_streams, "levels": levels,
            "cells": f"{w // cw}x{h // ch} of {cw}x{ch} px", "frames": n_frames,
            "max_motion_px": motion, "params": params_kw or {},
            "frames_per_s": n_streams * steps / total_s, "ms_per_step": 1000 * total_s / steps,
            "p50_ms": percentile(step_ms, 50), "p99_ms": percentile(step_ms, 99),
            "tracked_keypoints_per_s": float(st[..., 0].sum() + st[..., 1].sum()) / total_s,
            "survived_per_step": float(st[..., 2].sum() + st[..., 3].sum()) / steps,
            "tune": dict(zip(("k2_threads", "pyr_tile_shift", "pyr_first_levels", "k1_threads"),
                             tune))}


def batched_compare(torch, vio, steps, warmup, net, seqs=None):
    """The 16-stream batch, plain and with the learned initializer (trained
    gate, tracking from the proposal over levels 1..0, and the same network
    with the start at level 0): each step uploads one frame per stream into
    its slot (device to device, frames resident) and runs the batch's captured
    graph; per-step CUDA events give the step latency (every frame of a step
    completes with it). Steady state: the streams run `warmup` + 8 steps
    before the timed ones (no reset), as continuous streams do."""
    import numpy as np
    seqs = seqs or cfg4_frames()
    dev = [[torch.from_numpy(f).cuda() for f in cls] for cls in seqs]
    groups = []
    for (w, h, cw, ch) in CFG4_CLASSES:
        p = vio.default_params(n_levels=CFG4_LEVELS, cell_w=cw, cell_h=ch)
        groups.append((p, w, h, CFG4_STREAMS, 2 * (w // cw) * (h // ch)))
    n_streams = CFG4_STREAMS * len(CFG4_CLASSES)
    F = CFG4_FRAMES
    order = list(range(F)) + list(range(F - 2, 0, -1))   # forward and back: motion stays smooth
    res = {"streams": n_streams, "classes": [f"{w}x{h}" for (w, h, _, _) in CFG4_CLASSES],
           "levels": CFG4_LEVELS, "max_motion_px": CFG4_MOTION, "steps": steps,
           "timing": "steady state: warm-up steps, no reset before the timed steps"}
    start0 = net.cfg.start_level if net is not None else None
    modes = [("plain", None)]
    if net is not None:
        modes += [("learned", start0), ("learned_start0", 0)]
    for mode, start in modes:
        if net is not None:
            net.configure(start_level=start if start is not None else start0)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            b = vio.Batch(groups)
            if start is not None:
                b.set_initnet(net)

            def upload(t):
                for g in range(len(CFG4_CLASSES)):
                    for i in range(CFG4_STREAMS):
                        b.next_frame(g, i).copy_(dev[g][i][order[t % len(order)]],
                                                 non_blocking=True)

            for t in range(2):                 # frames in both slots for the autotuner
                upload(t)
                b.step(None, stream=s)
            tune_ms = b.autotune(reps=2, stream=s)
            b.set_graph(True)
            n_warm = warmup + 8
            for t in range(n_warm):
                upload(t)
                b.step(None, stream=s)
            s.synchronize()
            _, steps0 = b.read_stats(0)
            # a fixed 20 ms spin on the stream (~40M cycles at ~2 GHz) before
            # two more untimed steps: the host queues steps meanwhile, so the
            # early timed steps do not wait for a host that was descheduled
            # while it was only a step or two ahead
            torch.cuda._sleep(40_000_000)
            for t in range(n_warm, n_warm + 2):
                upload(t)
                b.step(None, stream=s)
            steps0 += 2
            n_warm += 2
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
            evs[0].record(s)
            for t in range(steps):
                upload(n_warm + t)
                b.step(None, stream=s)
                evs[t + 1].record(s)
            s.synchronize()
        lat = [evs[t].elapsed_time(evs[t + 1]) for t in range(steps)]
        total_s = evs[0].elapsed_time(evs[steps]) / 1000.0
        tracked = learned = survived = 0
        for g in range(len(CFG4_CLASSES)):
            st, n = b.read_stats(g)
            idx = [(steps0 + k) % vio.STATS_RING for k in range(steps)]
            a = st[idx].astype(np.int64)
            tracked += int(a[..., 0].sum() + a[..., 1].sum())
            survived += int(a[..., 2].sum() + a[..., 3].sum())
            learned += int(a[..., 7].sum())
        k2, shift, after, first, k1, dw = b.get_tune()
        slow = sorted(range(steps), key=lambda i: -lat[i])[:5]
        res[mode] = {"frames_per_s": n_streams * steps / total_s,
                     "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
                     "slowest_steps": [[i, round(lat[i], 4)] for i in slow],
                     "tracked_keypoints_per_s": tracked / total_s,
                     "survived_per_step": survived / steps,
                     "learned_share_of_survivors": learned / max(survived, 1),
                     "launches_per_step": b.launches_per_step(),
                     "start_level": start, "min_conf": net.cfg.min_conf if start is not None
                     else None,
                     "tune": {"k2_threads": k2, "pyr_tile_shift": shift,
                              "stereo_after_select": after, "pyr_first_levels": first,
                              "k1_threads": k1, "det_warps": dw, "best_ms": tune_ms}}
        b.close()
    if net is not None:
        net.configure(start_level=start0)
        for mode in ("learned", "learned_start0"):
            res[mode + "_vs_plain_fps"] = res[mode]["frames_per_s"] / res["plain"]["frames_per_s"]
            res[mode + "_vs_plain_p99"] = res[mode]["p99_ms"] / res["plain"]["p99_ms"]
        from paper_2609_30459_gb300 import initnet_train
        flat = [f for cls in seqs for f in cls[:1]]          # one stream of each size
        g = initnet_train.gain_eval(net, flat, n_levels=CFG4_LEVELS, cell=32,
                                    start_levels=(start0, 0), taus=(net.cfg.min_conf,))
        res["accuracy"] = {"sample": "one stream of each size, all frame pairs, 32x32 cells",
                           "keypoints": g["n"]}
        for mode, sl in (("learned", start0), ("learned_start0", 0)):
            res["accuracy"][mode] = g[f"start{sl}_tau{net.cfg.min_conf}"]
    return res


def serving_run(torch, vio, seconds, net, tune, seqs=None):
    """Config 5: 32 sessions (8 of each cfg-4 size) sending frames as Poisson
    processes of rate U[30, 200] Hz each for `seconds`, served by vio_server
    (device memory budget, continuous batching, learned start with the plain
    fallback). Frames come from pinned host memory (each session replays its
    sequence forward and back); latency is arrival -> completion seen by the
    server loop, which includes the upload, the queueing and the read-back."""
    import numpy as np
    from paper_2609_30459_gb300 import serving
    per_class = 8
    classes = []
    for (w, h, cw, ch) in CFG4_CLASSES:
        p = vio.default_params(n_levels=CFG4_LEVELS, cell_w=cw, cell_h=ch)
        classes.append((p, w, h, per_class, 2 * (w // cw) * (h // ch)))
    budget = 4 << 30                              # fixed device-memory budget
    slots, used = vio.server_plan(classes, budget)
    srv = vio.Server(classes, budget)
    if net is not None:
        srv.set_initnet(net)
    if tune is not None:
        srv.set_tune(*tune)
    seqs = seqs or cfg4_frames()
    pinned = [[torch.from_numpy(f).pin_memory() for f in cls] for cls in seqs]
    sessions, pools = [], []
    for c in range(len(CFG4_CLASSES)):
        for i in range(per_class):
            sid, adm = srv.open(c)
            sessions.append(sid)
            pools.append(pinned[c][i % len(pinned[c])])
    rng = np.random.default_rng(5000)
    rates = rng.uniform(30.0, 200.0, len(sessions))
    trace = serving.poisson_trace(rates, seconds, seed=5001)
    reqs = []
    for (t, i, k) in trace:
        pool = pools[i]
        reqs.append((sessions[i], t, pool[serving.pingpong(pool.shape[0], k)], k, 0))
    # warm-up: one frame per session (graph capture, first-frame detection)
    warm = [(sessions[i], 0.0, pools[i][0], -1, 0) for i in range(len(sessions))]
    srv.run_trace(warm, timeout_s=60.0)
    # the trace loop keeps its CPU: pinned to the core it starts on, at a
    # real-time priority where the system permits it
    srv.set_loop_policy(pin_cpu=-2, rt_priority=10)
    import gc
    gc.collect()
    gc.disable()                 # no collector pauses in the host process meanwhile
    time.sleep(1.0)
    t0 = time.perf_counter()
    try:
        done, steps = srv.run_trace(reqs, timeout_s=seconds + 120.0)
    finally:
        gc.enable()
    wall = time.perf_counter() - t0
    gap, n_gaps = srv.loop_stats()
    pinned_ok, rt_ok = srv.loop_policy_granted()
    summ = serving.latency_summary(done)
    srv.close_server()
    return {"sessions": len(sessions), "classes": [f"{w}x{h}" for (w, h, _, _) in CFG4_CLASSES],
            "rate_hz": "U[30,200] per session", "offered_fps": float(rates.sum()),
            "seconds": seconds, "requests": len(reqs), "steps": steps,
            "mean_batch": len(reqs) / max(steps, 1), "wall_s": wall,
            "budget_bytes": budget, "device_bytes": used, "slots": slots,
            "learned": net is not None,
            "host_loop": {"max_gap_ms": 1e3 * gap, "passes_over_1ms": n_gaps,
                          "pinned_cpu": pinned_ok, "realtime_priority": rt_ok,
                          "note": "the server's host loop polls continuously; a gap is time "
                                  "the process was not running (shared host CPUs)"},
            **summ}


def profile_frontend(w, h, n_streams, learned, steps=3):
    """A few frontend steps of one size (5 levels, cells for ~1000 keypoints
    per 1920x1080 image, motion up to 40 px), for kernel profiles."""
    import torch
    from paper_2609_30459_gb300 import initnet_train, synth, vio
    vio.load(build=True)
    cw, ch = {1920: (48, 43), 1280: (42, 36), 752: (37, 32)}.get(w, (32, 32))
    seq = synth.make_sequence(4012, steps, w, h, 1, max_motion=40.0, tex_size=2048)
    fr = torch.from_numpy(seq.frames).cuda()
    p = vio.default_params(n_levels=5, cell_w=cw, cell_h=ch)
    fe = vio.Frontend(p, w, h, n_streams, 2 * (w // cw) * (h // ch))
    net = vio.InitNet.load(initnet_train.DEFAULT_WEIGHTS) if learned else None
    if net is not None:
        fe.set_initnet(net)
    frames = fr.view(steps, 1, 2, h, w).expand(steps, n_streams, 2, h, w).contiguous()
    for t in range(steps):
        fe.step(frames[t])
    torch.cuda.synchronize()
    print(json.dumps({"profile_frontend": [w, h, n_streams], "learned": learned,
                      "tracks": int(fe.view()["track_count"].sum().item())}))
    return 0


def tune_frontend(torch, fe, frames5, combos, n=40, finalists=3, n_final=120):
    """Launch shapes of a frontend, timed on the path the bench times
    (`fe.run`, pipelined across frames): every candidate over frames5[3:3+n]
    after 3 warm-up frames, the better of two passes; the `finalists` fastest
    again over up to n_final frames, the best of three passes, so that a
    candidate that won one short pass by noise does not decide. frames5 is
    (frames, streams, 2, h, w). Returns (tune, ms per step)."""
    def timed(c, m, reps):
        fe.set_tune(*c)
        t = None
        for _ in range(reps):
            fe.reset()
            fe.run(frames5[:3])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fe.run(frames5[3:3 + m])
            e1.record()
            torch.cuda.synchronize()
            dt = e0.elapsed_time(e1) / m
            t = dt if t is None else min(t, dt)
        return t

    m1 = min(n, len(frames5) - 3)
    first = sorted(((timed(c, m1, 2), c) for c in combos), key=lambda x: x[0])
    m2 = min(n_final, len(frames5) - 3)
    final = sorted(((timed(c, m2, 3), c) for _, c in first[:finalists]), key=lambda x: x[0])
    best_t, best = final[0]
    fe.set_tune(*best)
    fe.reset()
    torch.cuda.synchronize()
    return best, best_t


def autotune_frontend(torch, fe, frames, n=40):
    import itertools
    frames5 = frames.view(N_FRAMES, 1, 2, H, W)
    combos = list(itertools.product((32, 64, 128, 256), (-1, 0, 1), (0, 1, 2), (128, 256)))
    best, best_t = tune_frontend(torch, fe, frames5, combos, n)
    return {"k2_threads": best[0], "pyr_tile_shift": best[1], "pyr_first_levels": best[2],
            "k1_threads": best[3], "ms_per_step": best_t}


def profile_pyramid_detect(n=512, reps=3):
    """vio_pyramid_detect of a device-resident batch of n images of the
    headline sequence, `reps` times (for launch lists and kernel profiles)."""
    import torch
    from paper_2609_30459_gb300 import synth, vio
    vio.load(build=True)
    seq = synth.make_sequence(2000, 4, W, H, 1, max_motion=MOTION, tex_size=2048)
    imgs = torch.from_numpy(seq.frames.reshape(-1, H, W)).cuda().repeat(n // 8, 1, 1)
    imgs = imgs.contiguous()
    p = vio.default_params(n_levels=LEVELS, cell_w=CELL_W, cell_h=CELL_H, k_per_cell=K_CELL)
    ctx = vio.Context(p, W, H, n)
    pyr = vio.Pyramids(imgs, LEVELS)
    cap = (W // CELL_W) * (H // CELL_H) * K_CELL
    kp = torch.empty((n, cap, 2), dtype=torch.float32, device="cuda")
    sc = torch.empty((n, cap), dtype=torch.int16, device="cuda")
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    for _ in range(reps):
        ctx.pyramid_detect(pyr, kp, sc, cnt, cap)
    torch.cuda.synchronize()
    print(json.dumps({"profile_pyramid_detect": n, "keypoints": int(cnt.sum().item())}))
    return 0


def profile_batch(mode, steps=18):
    """The 16-stream batch (cfg 4) stepped `steps` times without graphs, plain
    or with the learned start, so that every kernel is its own launch (for
    launch lists)."""
    import torch
    from paper_2609_30459_gb300 import initnet_train, vio
    vio.load(build=True)
    seqs = cfg4_frames()
    dev = [[torch.from_numpy(f).cuda() for f in cls] for cls in seqs]
    groups = []
    for (w, h, cw, ch) in CFG4_CLASSES:
        p = vio.default_params(n_levels=CFG4_LEVELS, cell_w=cw, cell_h=ch)
        groups.append((p, w, h, CFG4_STREAMS, 2 * (w // cw) * (h // ch)))
    order = list(range(CFG4_FRAMES)) + list(range(CFG4_FRAMES - 2, 0, -1))
    b = vio.Batch(groups)
    if mode == "learned":
        b.set_initnet(vio.InitNet.load(initnet_train.DEFAULT_WEIGHTS))
    b.set_tune(128, 0, 1, 2, 128)
    for t in range(steps):
        for g in range(len(CFG4_CLASSES)):
            for i in range(CFG4_STREAMS):
                b.next_frame(g, i).copy_(dev[g][i][order[t % len(order)]])
        b.step(None)
    torch.cuda.synchronize()
    print(json.dumps({"profile_batch": mode, "steps": steps}))
    b.close()
    return 0


def profile_initnet(n=1 << 16, reps=3):
    """The flow network's forward pass (vio_initnet_forward, tcgen05) on n
    random inputs with the shipped weights, `reps` times (kernel profiles)."""
    import torch
    from paper_2609_30459_gb300 import initnet_train, vio
    vio.load(build=True)
    net = vio.InitNet.load(initnet_train.DEFAULT_WEIGHTS)
    g = torch.Generator(device="cuda").manual_seed(11)
    x = (0.5 * torch.randn((n, 4, 16, 16), device="cuda", generator=g)).to(torch.bfloat16)
    x = x.view(torch.int16)
    out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    for _ in range(reps):
        net.forward(x, out)
    torch.cuda.synchronize()
    print(json.dumps({"profile_initnet": n, "status": vio.initnet_fault()}))
    return 0


def profile_detect(n=64, reps=3):
    """Standalone detection (vio_detect_grid) of a device-resident batch of n
    images of the headline sequence, pyramids built first, for kernel
    profiles."""
    import torch
    from paper_2609_30459_gb300 import synth, vio
    vio.load(build=True)
    seq = synth.make_sequence(2000, 4, W, H, 1, max_motion=MOTION, tex_size=2048)
    imgs = torch.from_numpy(seq.frames.reshape(-1, H, W)).cuda().repeat(n // 8, 1, 1)
    imgs = imgs.contiguous()
    p = vio.default_params(n_levels=LEVELS, cell_w=CELL_W, cell_h=CELL_H, k_per_cell=K_CELL)
    ctx = vio.Context(p, W, H, n)
    pyr = vio.Pyramids(imgs, LEVELS)
    ctx.pyramid_build(pyr)
    cap = (W // CELL_W) * (H // CELL_H) * K_CELL
    kp = torch.empty((n, cap, 2), dtype=torch.float32, device="cuda")
    sc = torch.empty((n, cap), dtype=torch.int16, device="cuda")
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    for _ in range(reps):
        ctx.detect_grid(pyr, pyr.batch(), kp, sc, cnt, cap)
    torch.cuda.synchronize()
    print(json.dumps({"profile_detect": n, "keypoints": int(cnt.sum().item())}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-frames", type=int, default=60)
    ap.add_argument("--batched-steps", type=int, default=300)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--profile-frontend", nargs=3, type=int, metavar=("W", "H", "STREAMS"),
                    help="only run 3 frontend steps of this size (for kernel profiles)")
    ap.add_argument("--learned", action="store_true", help="with --profile-frontend")
    ap.add_argument("--profile-pyramid-detect", type=int, nargs="?", const=512, default=None,
                    metavar="IMAGES",
                    help="only run vio_pyramid_detect 3 times on IMAGES images (default 512)")
    ap.add_argument("--profile-batch", choices=["plain", "learned"],
                    help="only step the 16-stream batch 18 times without graphs (launch lists)")
    ap.add_argument("--profile-initnet", type=int, nargs="?", const=1 << 16, default=None,
                    metavar="SAMPLES",
                    help="only run the network's forward pass 3 times on SAMPLES random inputs "
                         "(default 65536; for kernel profiles)")
    ap.add_argument("--profile-detect", type=int, nargs="?", const=64, default=None,
                    metavar="IMAGES",
                    help="only run 3 detections of a batch of IMAGES images (default 64; "
                         "for kernel profiles)")
    args = ap.parse_args()
    if args.profile_initnet:
        return profile_initnet(args.profile_initnet)
    if args.profile_detect:
        return profile_detect(args.profile_detect)
    if args.profile_batch:
        return profile_batch(args.profile_batch)
    if args.profile_pyramid_detect:
        return profile_pyramid_detect(args.profile_pyramid_detect)
    if args.profile_frontend:
        return profile_frontend(*args.profile_frontend, args.learned)
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

    # launch shapes of the frontend (results do not depend on them): every
    # combination timed over 40 frames, the fastest kept
    fe_tune = autotune_frontend(torch, fe, frames)

    # warm-up on the last frames of the sequence, then a fresh start at frame 0
    for i in range(args.warmup):
        fe.step(frames[N_FRAMES - args.warmup + i: N_FRAMES - args.warmup + i + 1])
    torch.cuda.synchronize()
    fe.reset()
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
    stats, steps_after = fe.read_stats()
    # per-stage times: a separate pass with CUDA events at every stage
    # boundary; per-step latency: another with only each step's first and
    # last event (events between launches cancel the tracking -> finalisation
    # overlap); steps in order, each after the previous one ended (the
    # throughput above is taken without events)
    n_lat = min(args.steps, 1000)

    def timed_pass(mode):
        fe.reset()
        fe.set_timing(mode)
        left = n_lat
        while left > 0:
            n = min(N_FRAMES, left)
            fe.run(frames5[:n])
            left -= n
        out = fe.read_timing(max_steps=n_lat)
        fe.set_timing(False)
        return out

    stage_ms, n_timed, stage_step_ms = timed_pass(1)
    _, _, step_ms = timed_pass(2)
    idx = [(steps_before + k) % vio.STATS_RING for k in range(args.steps)]
    st = stats[idx, 0, :].astype(np.int64)                       # (K, 7)
    tracked = int(st[:, 0].sum() + st[:, 1].sum())
    new_kp = int(st[:, 4].sum())
    stereo_in = int(st[:, 6].sum())                               # candidates matched
    survived = int(st[:, 2].sum() + st[:, 3].sum())

    t_max = total_s
    if world > 1:
        t_max = max_over_ranks(total_s, dist, "cuda")
    value = world * args.steps / t_max

    # tracking: latency/issue bound (one dependent Gauss-Newton chain per
    # keypoint and direction), so it is reported as keypoints per second and
    # its launch time, with the issue and stall counters of its ncu profile
    per_stage = {k: v / max(n_timed, 1) for k, v in stage_ms.items()}
    t_track = stage_ms["track"] / 1000.0 / max(n_timed, 1)
    tracking = {"kernel": "frame_track_kernel",
                "keypoints_per_launch": (tracked + stereo_in) / args.steps,
                "keypoint_tracks_per_s": (tracked + stereo_in) / args.steps / t_track,
                "avg_launch_us": 1e6 * t_track,
                "bound": "latency (dependent chains: 8 templates and 40 Gauss-Newton steps per "
                         "keypoint and direction)",
                "ncu": TRACK_NCU}

    # end to end through the C ABI from pinned host memory: every step uploads
    # its stereo pair and reads back the keypoint lists and new detections
    # (copy in, step, copy out, all enqueued). Throughput:
    # vio_frontend_step_host_async (pipelined across calls on the frontend's
    # streams) issued back to back over a ring of 4 frame and result slots, the
    # host waiting for (and reading) the results of the step two back.
    # Latency: vio_frontend_step_host with one host wait per frame.
    e2e = None
    if rank == 0 or world > 1:
        R = 4
        host = torch.from_numpy(frames_np).pin_memory()
        slots = torch.empty((R, 1, 2, H, W), dtype=torch.uint8, device="cuda")
        outs = [fe.host_outputs() for _ in range(R)]
        evs = [torch.cuda.Event() for _ in range(R)]
        for e in evs:
            e.record(stream)                           # creates the events
        counts = [o["count"].numpy() for o in outs]
        fe.reset()
        got = [0]

        def issue(k, pipelined):
            r = k % R
            f = k % N_FRAMES
            if pipelined:
                fe.step_host_async(host[f: f + 1], slots[r], outs[r], evs[r])
            else:
                fe.step_host(host[f: f + 1], slots[r], outs[r])
                evs[r].record(stream)

        def consume(k):
            evs[k % R].synchronize()
            got[0] += int(counts[k % R].sum())         # the host reads the result

        def run(n, sync_each):
            lat = []
            for k in range(n):
                ts = time.perf_counter()
                if not sync_each and k >= 2:
                    consume(k - 2)
                issue(k, not sync_each)
                if sync_each:
                    consume(k)
                    lat.append(time.perf_counter() - ts)
            if not sync_each:
                for k in range(max(n - 2, 0), n):
                    consume(k)
            return lat

        run(args.warmup, True)
        fe.reset()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        run(args.steps, False)
        e2e_s = time.perf_counter() - t0
        fe.reset()
        torch.cuda.synchronize()
        lat = run(min(args.steps, 1000), True)
        if world > 1:
            e2e_s = max_over_ranks(e2e_s, dist, "cuda")
        bo = sum(t.numel() * t.element_size() for t in outs[0].values())
        e2e = {"value": world * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 2 * H * W, "d2h_bytes_per_step": bo,
               "mode": "vio_frontend_step_host_async (pipelined on the frontend's streams) "
                       "issued back to back, results read two steps later",
               "sync_per_frame": {"frames_per_s": len(lat) / sum(lat),
                                  "p50_ms": 1000 * percentile(lat, 50),
                                  "p99_ms": 1000 * percentile(lat, 99)}}

    pd = pyramid_detect_roofline(torch, vio, frames, peaks, peak_src) if rank == 0 else None
    roofline = pd

    # config 3 (4 cameras = two stereo pairs at 1920x1080, motion up to 40 px)
    # and the paper's lite parameters on 752x480 sequences like the headline's
    extra_cfgs = None
    sel = None
    mbs = None
    lite = None
    if rank == 0 and not args.no_batched:
        # the cfg-3 frames (two stereo pairs of 1920x1080) as one detection batch
        from paper_2609_30459_gb300 import synth
        import numpy as np
        seqs3 = [synth.make_sequence(3000 + i, 100, 1920, 1080, 1, max_motion=40.0,
                                     tex_size=2048).frames for i in range(2)]
        sel = section("selection_variants", lambda: selection_variants(
            torch, vio, torch.from_numpy(np.stack(seqs3, 1)).cuda(), 1920, 1080, 5, 48, 43))
        del seqs3
        mbs = section("model_based_start", lambda: model_based_start(torch, vio))
        lite = section("lite_vs_standard", lambda: lite_vs_standard(torch, vio))
        extra_cfgs = [
            section("cfg3", lambda: frontend_config_run(
                torch, vio, "cfg3 high-pixel: 4 cameras (2 stereo pairs) 1920x1080, 100 frames, "
                "motion up to 40 px, 5 levels, 40x25 cells (1000 keypoints/image)", 1920, 1080,
                2, 5, 48, 43, 100, 40.0, 3000, args.batched_steps, roofline=(peaks, peak_src))),
            section("lite", lambda: frontend_config_run(
                torch, vio, "lite parameters (Sec. IV-D): minimum FAST threshold 20, 82-px "
                "cells, 3 Gauss-Newton iterations; 752x480, 4 levels", 752, 480, 1, 4, 82, 82,
                100, 15.0, 2000, args.batched_steps,
                params_kw={"gn_iters": 3, "thresholds": (40, 20)}))]

    # the 16 mixed-size sequences of cfg 4 (also the sessions' frames of cfg 5),
    # rendered once by a pool of host processes
    seqs4 = None
    if rank == 0 and not (args.no_batched and args.no_serve):
        seqs4 = cfg4_frames()
    batched = None
    if rank == 0 and not args.no_batched:
        from paper_2609_30459_gb300 import initnet_train
        net = None
        if os.path.exists(initnet_train.DEFAULT_WEIGHTS):
            net = vio.InitNet.load(initnet_train.DEFAULT_WEIGHTS)
        batched = section("batched_16_streams", lambda: batched_compare(
            torch, vio, args.batched_steps, args.warmup, net, seqs=seqs4))
        if net is not None and "error" not in batched:
            batched["initnet_tensor_roofline"] = section(
                "initnet_tensor_roofline",
                lambda: initnet_tensor_roofline(torch, vio, net, peaks, peak_src=peak_src))
    serve = None
    if rank == 0 and not args.no_serve:
        from paper_2609_30459_gb300 import initnet_train
        net = None
        if os.path.exists(initnet_train.DEFAULT_WEIGHTS):
            net = vio.InitNet.load(initnet_train.DEFAULT_WEIGHTS)
        # the batch's default tune: steps here hold one or two frames, for which
        # the fewest launches per step are best (the batched tune is for full steps)
        serve = section("serving_32_streams", lambda: serving_run(
            torch, vio, args.serve_seconds, net, None, seqs=seqs4))

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fps, cores, _ = oracle_frames_per_s(frames_np, args.cpu_frames)
        fps1, _, _ = oracle_frames_per_s(frames_np, 8, cores=1)
        cpu = {"value": fps, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_frames} consecutive frames of the same sequence through the "
                         f"FP64 oracle frontend (after 2 warm-up frames), tracking threaded "
                         f"over {cores} cores",
               "single_core": {"value": fps1, "unit": UNIT,
                               "sample": "8 frames after 2 warm-up frames, one thread"}}
        # oracle-side accuracy of the same configs (the oracle runs on the host
        # here, beside its timing)
        accuracy = section("accuracy", lambda: accuracy_report(torch, vio, frames_np))

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
            "e2e": e2e, "roofline": roofline, "tracking": tracking,
            "frontend_tune": fe_tune,
            "batched_16_streams": batched, "serving_32_streams": serve,
            "other_configs": extra_cfgs,
            "selection_variants": sel, "model_based_start": mbs,
            "lite_vs_standard": lite,
            "cpu_baseline": cpu, "accuracy": accuracy, "clocks": clk.summary(),
            "host_wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    fe.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
