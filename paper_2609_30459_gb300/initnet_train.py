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
import time

import numpy as np
import torch

from . import synth, vio

TRAIN_SEED0 = 900_000          # training sequences: seeds TRAIN_SEED0 + i
EVAL_SEED0 = 950_000           # held-out evaluation sequences


def _render(args):
    seed, n_frames, w, h, motion = args
    return synth.make_sequence(seed, n_frames, w, h, 1, max_motion=motion,
                               tex_size=2048).frames


def render_sequences(seeds, n_frames, w, h, motion, workers=0):
    """Frames (F, 2, h, w) uint8 of each seed, rendered on host cores (a
    spawned pool: no state of a CUDA context is inherited)."""
    jobs = [(s, n_frames, w, h, motion) for s in seeds]
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
          log=print, log_every=200, eval_set=None):
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
                                   1.0 / batch, grad, loss)
            net.step += 1
            vio.initnet_adam(net.master, grad, net.m, net.v, net.step, rate)
            if i % log_every == 0 or i == steps - 1:
                hist.append((i, loss.item() / batch))
                msg = ""
                if eval_set is not None:
                    net.pack()
                    ev = evaluate(net, *eval_set)
                    msg = (f" | held-out within 1px {ev['within_1px']:.3f} median "
                           f"{ev['median_err_px']:.2f}px gated0.5 {ev['gated_0.5']:.3f} "
                           f"({ev['gated_0.5_within_1px']:.3f})")
                log(f"  step {i}/{steps} loss {hist[-1][1]:.4f} lr {rate:.2e} "
                    f"({time.time() - t0:.1f}s){msg}")
    net.pack()
    torch.cuda.synchronize()
    return hist


@torch.no_grad()
def evaluate(net: vio.InitNet, X, F, chunk=65536):
    """Fraction of proposals within 1 and 2 px of the target, mean confidence
    of each group, and the within-1px fraction among confident proposals."""
    outs = [net.forward(X[i:i + chunk]) for i in range(0, len(X), chunk)]
    o = torch.cat(outs)
    err = torch.linalg.norm(o[:, :2] - F, dim=1)
    conf = o[:, 2]
    good = err < 1.0
    res = {"n": len(X), "within_1px": good.float().mean().item(),
           "within_2px": (err < 2.0).float().mean().item(),
           "median_err_px": err.median().item(),
           "zero_start_within_1px": (torch.linalg.norm(F, dim=1) < 1.0).float().mean().item()}
    for tau in (0.3, 0.5, 0.7, 0.9):
        m = conf >= tau
        res[f"gated_{tau}"] = m.float().mean().item()
        res[f"gated_{tau}_within_1px"] = good[m].float().mean().item() if m.any() else 0.0
    return res


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
    net = vio.InitNet(he_init(0), a.level_a, a.level_b, a.start_level, a.min_conf)
    print("before:", evaluate(net, Xe, Fe))
    train(net, X, F, epochs=a.epochs, batch=a.batch, lr=a.lr, log_every=a.log_every,
          eval_set=(Xe, Fe))
    ev = evaluate(net, Xe, Fe)
    print("held-out:", ev)
    net.save(a.out)
    print(f"saved {a.out} after {time.time() - t0:.0f}s")
    return ev


if __name__ == "__main__":
    main()
