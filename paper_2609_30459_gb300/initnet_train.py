"""Training of the learned flow initializer, on the GPU through the library's
own kernels (no autograd): samples from the plain tracker, then minibatch
Adam over them.

Samples. Synthetic stereo sequences (the generator of ``synth``), per
camera and consecutive frame pair: grid-cell detection on the earlier frame,
the plain pyramidal KLT with the forward-backward check (Sec. III-E) into
the later frame; every keypoint it tracks with status OK gives one sample:
the network input at levels (level_a, level_b) around the keypoint, and the
tracked flow as the target. The sequences' seeds are disjoint from those of
the tests and the benchmark.

Command line:
    python -m paper_2609_30459_gb300.initnet_train --out weights.npz
"""
from __future__ import annotations

import argparse
import math
import multiprocessing as mp
import os
import time

import numpy as np
import torch

from . import synth, vio

DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data",
                               "initnet.npz")
TRAIN_SEED0 = 900_000          # training sequences: seeds TRAIN_SEED0 + i
EVAL_SEED0 = 950_000           # held-out evaluation sequences


def _render(args):
    seed, n_frames, w, h, motion, whole = args
    seq = synth.make_sequence(seed, n_frames, w, h, 1, max_motion=motion, tex_size=2048)
    return seq if whole else seq.frames


def render_sequences(seeds, n_frames, w, h, motion, workers=0, whole=False):
    """Frames (F, 2, h, w) uint8 of each seed (or the whole synth.Sequence),
    rendered on host cores (a spawned pool: no state of a CUDA context is
    inherited)."""
    jobs = [(s, n_frames, w, h, motion, whole) for s in seeds]
    if workers <= 1:
        return [_render(j) for j in jobs]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        return pool.map(_render, jobs)


def samples_from_frames(frames, level_a, level_b, n_levels=5, cell=16, device="cuda"):
    """(x int16 [n,4,16,16] BF16 bits, flow float32 [n,2]) from one sequence."""
    F, _, h, w = frames.shape
    p = vio.default_params(n_levels=n_levels, cell_w=cell, cell_h=cell)
    cap = (w // cell) * (h // cell)
    ctx = vio.Context(p, w, h, F)
    xs, fs = [], []
    for cam in range(2):
        lv0 = torch.from_numpy(np.ascontiguousarray(frames[:, cam])).to(device)
        pyr = vio.Pyramids(lv0, n_levels)
        kp = torch.empty((F, cap, 2), dtype=torch.float32, device=device)
        sc = torch.empty((F, cap), dtype=torch.int16, device=device)
        cnt = torch.empty(F, dtype=torch.int32, device=device)
        ctx.pyramid_detect(pyr, kp, sc, cnt, cap)
        src, dst = pyr.batch(0, 1, F - 1), pyr.batch(1, 1, F - 1)
        pts = kp[: F - 1].contiguous()
        c = cnt[: F - 1].contiguous()
        out = torch.empty((F - 1, cap, 3), dtype=torch.float32, device=device)
        st = torch.empty((F - 1, cap), dtype=torch.uint8, device=device)
        ctx.track_patches(pyr, src, dst, pts, c, cap, out, st)
        x = torch.empty((F - 1, cap, 4, 16, 16), dtype=torch.int16, device=device)
        vio.initnet_extract(pyr, src, dst, pts, c, cap, level_a, level_b, x)
        ok = st == vio.TRACK_STATUS["OK"]
        xs.append(x[ok])
        fs.append((out[..., :2] - pts)[ok])
    ctx.close()
    return torch.cat(xs), torch.cat(fs)


def build_dataset(n_samples, seeds_from, level_a=2, level_b=3, w=640, h=480, n_frames=21,
                  motion=40.0, workers=8, device="cuda", log=print):
    xs, fs, n, k = [], [], 0, 0
    batch = max(workers, 1)
    while n < n_samples:
        seeds = [seeds_from + k + i for i in range(batch)]
        k += batch
        t0 = time.time()
        seqs = render_sequences(seeds, n_frames, w, h, motion, workers)
        t1 = time.time()
        for fr in seqs:
            x, f = samples_from_frames(fr, level_a, level_b, device=device)
            xs.append(x)
            fs.append(f)
            n += len(x)
        log(f"  {n} samples ({k} sequences; render {t1 - t0:.1f}s, "
            f"track {time.time() - t1:.1f}s)")
    return torch.cat(xs)[:n_samples].contiguous(), torch.cat(fs)[:n_samples].contiguous()


def he_init(seed=0):
    """He-normal weights, zero biases, in the master layout."""
    g = np.random.default_rng(seed)
    fan = [("w1", 32 * 36, 36), ("b1", 32, 0), ("w2", 32 * 288, 288), ("b2", 32, 0),
           ("w3", 32 * 288, 288), ("b3", 32, 0), ("w4", 64 * 128, 128), ("b4", 64, 0),
           ("w5", 3 * 64, 64), ("b5", 3, 0)]
    parts = [g.normal(0, math.sqrt(2.0 / f), n) if f else np.zeros(n) for _, n, f in fan]
    flat = np.concatenate(parts).astype(np.float32)
    assert flat.size == vio.INITNET_N_PARAMS
    return flat


def train(net: vio.InitNet, X, F, epochs=2, batch=1024, lr=2e-3, lr_min=1e-4, seed=0,
          log=print, log_every=200, eval_set=None, label_radius=1.0):
    """Minibatch Adam; the learning rate decays by a cosine from lr to lr_min."""
    N = len(X)
    dev = X.device
    if net.m is None:
        net.m = torch.zeros_like(net.master)
        net.v = torch.zeros_like(net.master)
    grad = torch.zeros_like(net.master)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    steps = epochs * (N // batch)
    hist = []
    t0 = time.time()
    for e in range(epochs):
        perm = torch.randperm(N, generator=gen).to(torch.int32).to(dev)
        for b in range(N // batch):
            i = e * (N // batch) + b
            rate = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * i / max(steps, 1)))
            net.pack()
            grad.zero_()
            loss.zero_()
            vio.initnet_train_step(net.packed, X, F, perm[b * batch:(b + 1) * batch], batch,
                                   1.0 / batch, grad, loss, label_radius=label_radius)
            net.step += 1
            vio.initnet_adam(net.master, grad, net.m, net.v, net.step, rate)
            if i % log_every == 0 or i == steps - 1:
                hist.append((i, loss.item() / batch))
                msg = ""
                if eval_set is not None:
                    net.pack()
                    ev = evaluate(net, *eval_set, radius=label_radius)
                    msg = (f" | held-out within 1px {ev['within_1px']:.3f} median "
                           f"{ev['median_err_px']:.2f}px gated0.5 {ev['gated_0.5']:.3f} "
                           f"({ev['gated_0.5_within_r']:.3f})")
                log(f"  step {i}/{steps} loss {hist[-1][1]:.4f} lr {rate:.2e} "
                    f"({time.time() - t0:.1f}s){msg}")
    net.pack()
    torch.cuda.synchronize()
    return hist


@torch.no_grad()
def evaluate(net: vio.InitNet, X, F, chunk=65536, radius=1.0):
    """Fraction of proposals within 1, 2 and r px of the target, and per
    confidence gate the fraction gated and the within-r fraction among them."""
    outs = [net.forward(X[i:i + chunk]) for i in range(0, len(X), chunk)]
    o = torch.cat(outs)
    err = torch.linalg.norm(o[:, :2] - F, dim=1)
    conf = o[:, 2]
    good = err < radius
    res = {"n": len(X), "within_1px": (err < 1.0).float().mean().item(),
           "within_2px": (err < 2.0).float().mean().item(),
           "within_r": good.float().mean().item(),
           "median_err_px": err.median().item(),
           "zero_start_within_1px": (torch.linalg.norm(F, dim=1) < 1.0).float().mean().item()}
    for tau in (0.3, 0.5, 0.7, 0.9):
        m = conf >= tau
        res[f"gated_{tau}"] = m.float().mean().item()
        res[f"gated_{tau}_within_r"] = good[m].float().mean().item() if m.any() else 0.0
    return res


def true_flow(seq, cam, t, pts):
    """Ground-truth positions in frame t+1 of points of frame t, camera cam
    (0 left, 1 right) of a generated sequence (synth.Sequence)."""
    h, w = seq.frames.shape[2:]
    d0, d1 = seq.disparity
    P = np.asarray(pts, np.float64).reshape(-1, 2).copy()
    if cam == 1:                       # right pixel (x, y) sees left pixel (x + d(y), y)
        P[:, 0] += d0 + d1 * P[:, 1] / h
    Q = synth.PlanarScene.map_points(seq.poses[t][0], seq.poses[t + 1][0], P, w, h, seq.c_tex)
    if cam == 1:
        Q[:, 0] -= d0 + d1 * Q[:, 1] / h
    return Q


@torch.no_grad()
def gain_eval(net: vio.InitNet, frames_list, n_levels=5, cell=32, start_levels=(1, 2),
              taus=(0.1, 0.3, 0.5, 0.7), tol=1e-3, truth_px=0.5, device="cuda"):
    """What the network gains over the plain tracker, per (start level, gate):
    on each sequence, per camera and frame pair, detection on the earlier
    frame, then the plain track (whole pyramid, zero start) and the track
    from the proposal over levels start..0, both with the forward-backward
    check. Reports the fraction of keypoints gated, the fraction of gated
    tracks that end OK and converged (the network's max_last_step gate), the
    fraction of those within `tol` px of the plain result where the plain
    track is OK, and where it has also converged, the tracks the plain track loses
    but the proposal keeps, and the mean number of pyramid levels tracked
    per keypoint (plain: n_levels; learned: start+1, plus n_levels on a
    fallback). With generated sequences (synth.Sequence) instead of frame
    arrays, also the fraction of plain-OK and of gained tracks within
    truth_px of the ground truth."""
    OKS = vio.TRACK_STATUS["OK"]
    acc = {}
    n_total = 0
    for item in frames_list:
        seq = item if hasattr(item, "poses") else None
        frames = seq.frames if seq is not None else item
        F, _, h, w = frames.shape
        p = vio.default_params(n_levels=n_levels, cell_w=cell, cell_h=cell)
        cap = (w // cell) * (h // cell)
        ctx = vio.Context(p, w, h, F)
        for cam in range(2):
            lv0 = torch.from_numpy(np.ascontiguousarray(frames[:, cam])).to(device)
            pyr = vio.Pyramids(lv0, n_levels)
            kp = torch.empty((F, cap, 2), dtype=torch.float32, device=device)
            sc = torch.empty((F, cap), dtype=torch.int16, device=device)
            cnt = torch.empty(F, dtype=torch.int32, device=device)
            ctx.pyramid_detect(pyr, kp, sc, cnt, cap)
            src, dst = pyr.batch(0, 1, F - 1), pyr.batch(1, 1, F - 1)
            pts = kp[: F - 1].contiguous()
            c = cnt[: F - 1].contiguous()
            out_p = torch.empty((F - 1, cap, 3), dtype=torch.float32, device=device)
            st_p = torch.empty((F - 1, cap), dtype=torch.uint8, device=device)
            ls_p = torch.empty((F - 1, cap), dtype=torch.float32, device=device)
            ctx.track_patches(pyr, src, dst, pts, c, cap, out_p, st_p, last_step=ls_p)
            x = torch.empty((F - 1, cap, 4, 16, 16), dtype=torch.int16, device=device)
            vio.initnet_extract(pyr, src, dst, pts, c, cap, net.cfg.level_a, net.cfg.level_b, x)
            prop = net.forward(x.view(-1, 4, 16, 16)).view(F - 1, cap, 3)
            init = torch.zeros((F - 1, cap, 3), dtype=torch.float32, device=device)
            init[..., :2] = pts + prop[..., :2]
            valid = st_p != vio.TRACK_STATUS["EMPTY"]
            n_total += int(valid.sum())
            truth = None
            if seq is not None:
                pts_h = pts.cpu().numpy()
                truth = torch.from_numpy(np.stack([true_flow(seq, cam, t, pts_h[t])
                                                   for t in range(F - 1)]).astype(np.float32))
                truth = truth.to(device).view(F - 1, cap, 2)
                e_p = torch.linalg.norm(out_p[..., :2] - truth, dim=-1)
            gate_step = net.cfg.max_last_step
            for s in start_levels:
                out_l = torch.empty_like(out_p)
                st_l = torch.empty_like(st_p)
                ls_l = torch.empty_like(ls_p)
                ctx.track_patches(pyr, src, dst, pts, c, cap, out_l, st_l, init=init,
                                  from_level=s, last_step=ls_l)
                d = torch.linalg.norm(out_l[..., :2] - out_p[..., :2], dim=-1)
                # a learned track counts when it ends OK and has converged (its
                # last level-0 step within the gate); the plain result "succeeds"
                # when it ends OK, and is settled when it has converged too
                conv_l = (ls_l <= gate_step) if gate_step > 0 else torch.ones_like(st_l, dtype=torch.bool)
                conv_p = (ls_p <= gate_step) if gate_step > 0 else torch.ones_like(st_p, dtype=torch.bool)
                for tau in taus:
                    g = valid & (prop[..., 2] >= tau)
                    lok = g & (st_l == OKS) & conv_l
                    pok = valid & (st_p == OKS)
                    both = lok & pok
                    both_conv = both & conv_p
                    k = (s, tau)
                    a = acc.setdefault(k, dict(gated=0, learned_ok=0, both=0, agree=0, gained=0,
                                               plain_ok=0, levels=0.0, plain_true=0,
                                               gained_true=0, truth=False, both_conv=0,
                                               agree_conv=0))
                    a["both_conv"] += int(both_conv.sum())
                    a["agree_conv"] += int((both_conv & (d < tol)).sum())
                    if truth is not None:
                        e_l = torch.linalg.norm(out_l[..., :2] - truth, dim=-1)
                        a["truth"] = True
                        a["plain_true"] += int((pok & (e_p < truth_px)).sum())
                        a["gained_true"] += int((lok & ~pok & (e_l < truth_px)).sum())
                    a["gated"] += int(g.sum())
                    a["learned_ok"] += int(lok.sum())
                    a["both"] += int(both.sum())
                    a["agree"] += int((both & (d < tol)).sum())
                    a["gained"] += int((lok & ~pok).sum())
                    a["plain_ok"] += int(pok.sum())
                    a["levels"] += float((s + 1) * g.sum() + n_levels * (valid & ~lok).sum())
        ctx.close()
    out = {"n": n_total, "n_levels": n_levels}
    for (s, tau), a in acc.items():
        out[f"start{s}_tau{tau}"] = {
            "gated": a["gated"] / max(n_total, 1),
            "learned_ok_of_gated": a["learned_ok"] / max(a["gated"], 1),
            "agree_of_both_ok": a["agree"] / max(a["both"], 1),
            "agree_where_plain_converged": a["agree_conv"] / max(a["both_conv"], 1),
            "plain_converged_of_both_ok": a["both_conv"] / max(a["both"], 1),
            "gained": a["gained"], "plain_ok": a["plain_ok"],
            "levels_per_kp": a["levels"] / max(n_total, 1)}
        if a["truth"]:
            out[f"start{s}_tau{tau}"].update(
                plain_ok_within_truth=a["plain_true"] / max(a["plain_ok"], 1),
                gained_within_truth=a["gained_true"] / max(a["gained"], 1))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--samples", type=int, default=1_000_000)
    ap.add_argument("--eval-samples", type=int, default=50_000)
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--level-a", type=int, default=2)
    ap.add_argument("--level-b", type=int, default=3)
    ap.add_argument("--start-level", type=int, default=1)
    ap.add_argument("--min-conf", type=float, default=0.5)
    ap.add_argument("--motion", type=float, default=40.0)
    ap.add_argument("--log-every", type=int, default=1000)
    ap.add_argument("--label-radius", type=float, default=3.0)
    ap.add_argument("--gain-seqs", type=int, default=4)
    ap.add_argument("--resume", default=None, help="checkpoint to continue training from")
    a = ap.parse_args(argv)
    # the render pool is spawned before the first CUDA call
    t0 = time.time()
    vio.load()
    print(f"building {a.samples} training samples")
    X, F = build_dataset(a.samples, TRAIN_SEED0, a.level_a, a.level_b, motion=a.motion,
                         workers=a.workers)
    print(f"building {a.eval_samples} held-out samples")
    Xe, Fe = build_dataset(a.eval_samples, EVAL_SEED0, a.level_a, a.level_b, motion=a.motion,
                           workers=a.workers)
    print(f"data ready in {time.time() - t0:.0f}s; |flow| mean "
          f"{torch.linalg.norm(F, dim=1).mean().item():.2f} px")
    if a.resume:      # weights, Adam moments and step count of a checkpoint
        net = vio.InitNet.load(a.resume)
        net.configure(level_a=a.level_a, level_b=a.level_b, start_level=a.start_level,
                      min_conf=a.min_conf)
    else:
        net = vio.InitNet(he_init(0), a.level_a, a.level_b, a.start_level, a.min_conf)
    print("before:", evaluate(net, Xe, Fe, radius=a.label_radius))
    train(net, X, F, epochs=a.epochs, batch=a.batch, lr=a.lr, log_every=a.log_every,
          eval_set=(Xe, Fe), label_radius=a.label_radius)
    ev = evaluate(net, Xe, Fe, radius=a.label_radius)
    print("held-out:", ev)
    net.save(a.out, label_radius=a.label_radius, samples=a.samples, epochs=a.epochs,
             motion_px=a.motion, seed0=TRAIN_SEED0)
    print(f"saved {a.out} after {time.time() - t0:.0f}s")
    if a.gain_seqs > 0:
        seqs = render_sequences([EVAL_SEED0 + 500 + i for i in range(a.gain_seqs)], 21, 640,
                                480, a.motion, a.workers, whole=True)
        gain = gain_eval(net, seqs)
        for k, v in gain.items():
            print(f"gain {k}: {v}")
    return ev


if __name__ == "__main__":
    main()
