"""The pyramid, detection, tracker and tensor-core network device code run
on the host (no GPU) under AddressSanitizer, against the oracle: the check
that stands in for a bounds checking build and for compute-sanitizer, which
is closed on the GPU pool.

tests/emu/blockemu.h emulates thread blocks with one host thread per CUDA
thread and real barriers for __syncthreads, named barriers and the warp
collectives; the harnesses give every CTA's shared memory a heap buffer of
exactly its computed size (and the pyramid's launch size must cover every
tile's plan), so any out-of-bounds shared or global access, any wrong
keypoint, pyramid value or network output, and any collective called from
divergent lanes (a deadlock the emulator reports) fails the test. The device
headers are compiled unchanged except for two host spellings: the named
barrier's inline PTX becomes an emulated barrier, and a function-scope
__shared__ variable a block-shared static (blocks run one at a time). The
network's tcgen05 primitives (tc05.cuh) are replaced by tests/emu/tc05_emu.h,
which carries out each MMA through its decoded shared-memory descriptors (so
the operand layouts of the kernel are what is checked) into an emulated
tensor memory."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import initnet as onet

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2609_30459_gb300", "csrc")
EMU = os.path.join(ROOT, "tests", "emu")
PYR_DETECT = os.path.join(ROOT, "oracle", "src", "pyramid_detect.cpp")


def _host_copy(dst):
    shutil.copy(os.path.join(EMU, "tc05_emu.h"), os.path.join(dst, "tc05.cuh"))
    for name in ("common.cuh", "pyramid_dev.cuh", "detect_dev.cuh", "initnet_dev.cuh",
                 "initnet_tc.cuh", "track_dev.cuh", "frame.cuh", "finalize_dev.cuh",
                 "initnet_train_dev.cuh"):
        s = open(os.path.join(CSRC, name)).read()
        s = re.sub(r'asm volatile\("bar\.sync (\d), %0;" ::"r"\(n\) : "memory"\);',
                   r"emu_bar(\1, n);", s)
        s = s.replace("__shared__ PassPlan plan;", "static PassPlan plan;")
        s = s.replace("__shared__ int learned_s;", "static int learned_s;")
        s = re.sub(r'asm volatile\(\s*"mma\.sync\.aligned\.m16n8k16.*?\);',
                   "emu_mma16816(d, a, b0, b1);", s, flags=re.S)
        open(os.path.join(dst, name), "w").write(s)


def _build(tmp_path, main, extra=()):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    cuda_inc = "/usr/local/cuda/include"
    if not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("no CUDA headers")
    _host_copy(str(tmp_path))
    exe = str(tmp_path / (main + ".bin"))
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fsanitize=address", "-pthread",
           "-I", str(tmp_path), "-I", EMU, "-I", cuda_inc, "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "oracle", "src"), "-o", exe, os.path.join(EMU, main + ".cpp"),
           *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("AddressSanitizer not available")
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def _run(exe, *args, timeout=600, expect="FAILS 0"):
    r = subprocess.run([exe, *map(str, args)], capture_output=True, text=True, timeout=timeout,
                       env={**os.environ, "ASAN_OPTIONS": "detect_leaks=0"})
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    if expect:
        assert expect in out, out[-4000:]
    return out


def test_pyramid_pass_on_host(tmp_path):
    oracle.build()
    out = _run(_build(tmp_path, "pyr_check", [PYR_DETECT]))
    assert re.search(r"cases (\d+)", out) and int(re.search(r"cases (\d+)", out).group(1)) > 30


def test_detection_on_host(tmp_path):
    oracle.build()
    _run(_build(tmp_path, "det_check", [PYR_DETECT]))


def _bf16_bits(a):
    return (np.ascontiguousarray(onet.bf16_round(a), np.float32).view(np.uint32) >> 16
            ).astype(np.uint16)


def _packed(p):
    """The packed weights of vio_initnet_pack: BF16 [N][K] rows (conv K =
    c*9 + u*3 + v, conv1 padded to 48, fc2 to 8 rows), then 168 FP32 biases."""
    w1 = np.zeros((32, 48))
    w1[:, :36] = p["w1"].reshape(32, 36)
    w5 = np.zeros((8, 64))
    w5[:3] = p["w5"]
    w = np.concatenate([_bf16_bits(m).reshape(-1) for m in
                        (w1, p["w2"].reshape(32, 288), p["w3"].reshape(32, 288), p["w4"], w5)])
    b = np.zeros(168, np.float32)
    b[0:32], b[32:64], b[64:96], b[96:160], b[160:163] = p["b1"], p["b2"], p["b3"], p["b4"], p["b5"]
    return w.tobytes() + b.tobytes()


@pytest.mark.parametrize("n,blocks", [(70, 2), (32, 1)])
def test_initnet_tc_forward_on_host(tmp_path, n, blocks):
    """Rounds of 32 over a persistent grid (a ragged last round, a zero input)
    against the FP64 oracle with BF16 activations, at the GPU test's bound."""
    rng = np.random.default_rng(n)
    fan = {"w1": 36, "w2": 288, "w3": 288, "w4": 128, "w5": 64}
    p = {k: (rng.normal(0, np.sqrt(2.0 / fan[k]), onet.SHAPES[k]) if k.startswith("w")
             else rng.normal(0, 0.05, onet.SHAPES[k])) for k in onet.ORDER}
    p = onet.unflatten(onet.flatten(p).astype(np.float32).astype(np.float64))
    x = (rng.integers(0, 256, (n, 4, 16, 16)).astype(np.float64) - 128) / 64
    x[min(3, n - 1)] = 0
    xb = (x.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    inp, outp = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        f.write(np.array([n, blocks], np.int32).tobytes())
        f.write(_packed(p))
        f.write(xb.tobytes())
    _run(_build(tmp_path, "net_check"), inp, outp, expect=None)
    got = np.fromfile(outp, np.float32).reshape(n, 3).astype(np.float64)
    pb = {k: (onet.bf16_round(v) if k.startswith("w") else v) for k, v in p.items()}
    o = np.array([onet.forward(pb, xi, act_bf16=True) for xi in x])
    exp = np.stack([o[:, 0] * 16, o[:, 1] * 16, onet.sigmoid(o[:, 2])], 1)
    err = np.abs(got - exp)
    tol = 4e-3   # the GPU forward test's bound on the raw outputs (BF16 rounding flips)
    assert np.all(err[:, :2] <= 16 * tol), err.max(0)
    assert np.all(err[:, 2] <= tol / 4), err.max(0)
    assert np.median(err[:, :2]) < 16 * 1e-4


def test_tracker_on_host(tmp_path):
    """The tracker's device code (templates, branch-free Gauss-Newton steps
    with clamped reads, the forward-backward check) on the host, every
    pyramid level between poisoned gaps so that AddressSanitizer reports any
    read outside a level, against the FP64 oracle at the GPU parity tests'
    bounds: detected keypoints, keypoints at and beyond the borders, starts
    near the answer and far from it."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import parity_util
    from paper_2609_30459_gb300 import synth
    oracle.build()
    w, h, L, iters, fbm = 200, 152, 3, 5, 0.5
    seq = synth.make_sequence(7100, 2, w, h, 1, max_motion=6.0, tex_size=1024)
    src = oracle.pyramid(seq.frames[0, 0], L)
    dst = oracle.pyramid(seq.frames[1, 0], L)
    det, _ = oracle.detect_grid(seq.frames[0, 0], 25, 19, k=1)
    border = np.array([[1, 1], [3, 70], [195, 70], [100, 149], [100.5, 2.25], [198.9, 150.9],
                       [12.25, 12.75], [187.5, 139.5], [7.5, 70], [8.0, 40], [70, 7.5],
                       [189.5, 100], [100, 141.5]], np.float32)
    pts = np.concatenate([det, border]).astype(np.float32)
    plain = oracle.track(src, dst, pts, gn_iters=iters, fb_max_dist=fbm)
    # starts: the plain answer (a start at the optimum) for the first eight
    # detections and a start 11 px off for the next eight
    m = len(det)
    init = np.zeros((len(pts), 3), np.float32)
    has = np.zeros(len(pts), bool)
    init[:8, :2] = plain["warp"][:8, :2]
    has[:8] = plain["status"][:8] == 0
    init[8:16, :2] = pts[8:16] + np.array([9.0, -7.0], np.float32)
    has[8:16] = True
    cases = [(pts, None, np.zeros(len(pts), bool)),
             (pts[:16][has[:16]], init[:16][has[:16]], np.ones(int(has[:16].sum()), bool))]
    inp, outp = tmp_path / "in.bin", tmp_path / "out.bin"
    exe = _build(tmp_path, "trk_check")
    compared = 0
    for P, ini, flag in cases:
        with open(inp, "wb") as f:
            f.write(np.array([L, len(P), iters], np.int32).tobytes())
            f.write(np.array([fbm], np.float32).tobytes())
            for l in range(L):
                f.write(np.array(src[l].shape[::-1], np.int32).tobytes())
                f.write(np.ascontiguousarray(src[l], np.uint8).tobytes())
                f.write(np.ascontiguousarray(dst[l], np.uint8).tobytes())
            rec = np.zeros((len(P), 5), np.float32)
            rec[:, :2] = P
            if ini is not None:
                rec[:, 2:4] = ini[:, :2]
            rec[:, 4] = flag
            f.write(rec.tobytes())
        _run(exe, inp, outp, timeout=900, expect="points")
        got = np.fromfile(outp, np.float32).reshape(-1, 5)
        ref = oracle.track(src, dst, P, init=ini, gn_iters=iters, fb_max_dist=fbm)
        st = parity_util.compare_tracks(got[:, 1:3], got[:, 0].astype(np.uint8), ref, fbm,
                                        g_theta=got[:, 3])
        compared += len(P)
        assert (got[:, 0] == 0).sum() >= len(P) // 3, got[:, 0]
    assert compared >= m + 8


def _finalize_expected(W, H, cw, ch, k, cap, n0, n1, next_id, have_prev, trk_status, trk_xy,
                       list_id, cand_count, cand, spec_status, spec_xy):
    """One stream's finalisation written from its rules (Sec. III-B/III-D:
    surviving tracks in order, cell occupancy of camera 0's survivors, per
    cell in raster order the first k - occupancy candidates, new ids in
    selection order, camera 1 gets the successful stereo matches of the new
    keypoints, lists truncated to the capacity)."""
    from oracle import frontend as ofe
    gx, gy = W // cw, H // ch
    n0, n1 = (min(n0, cap), min(n1, cap)) if have_prev else (0, 0)
    ok0 = [i for i in range(n0) if trk_status[i] == 0]
    ok1 = [i for i in range(n1) if trk_status[cap + i] == 0]
    xy0 = [trk_xy[i] for i in ok0]
    xy1 = [trk_xy[cap + i] for i in ok1]
    id0 = [list_id[i] for i in ok0]
    id1 = [list_id[cap + i] for i in ok1]
    occ = ofe.occupancy(np.array(xy0, np.float32).reshape(-1, 2), W, H, cw, ch).reshape(-1)
    new_xy, new_m = [], []
    for cell in range(gx * gy):
        nsel = max(0, min(k - min(int(occ[cell]), 255), int(cand_count[cell])))
        for r in range(nsel):
            q = cell * k + r
            idx = (~int(cand[q])) & 0xffffffff
            new_xy.append([float(idx % W), float(idx // W)])
            if spec_status[q] == 0:
                new_m.append((len(new_xy) - 1, spec_xy[q]))
    ids = [next_id + o for o in range(len(new_xy))]
    cam0_xy = (xy0 + new_xy)[:cap]
    cam0_id = (id0 + ids)[:cap]
    cam1_xy = (xy1 + [m[1] for m in new_m])[:cap]
    cam1_id = (id1 + [ids[m[0]] for m in new_m])[:cap]
    return {"count": [len(cam0_xy), len(cam1_xy)], "xy": [cam0_xy, cam1_xy],
            "id": [cam0_id, cam1_id], "new_xy": new_xy[:cap], "new_count": min(len(new_xy), cap),
            "next_id": next_id + len(new_xy), "occ": np.minimum(occ, 255),
            "stats": [n0, n1, len(ok0), len(ok1), len(new_xy), len(new_m),
                      int(np.sum(cand_count)), 0]}


@pytest.mark.parametrize("case", ["one_pass", "first_frame", "truncated", "multi_pass"])
def test_finalize_on_host(tmp_path, case):
    """The finalisation's device code on the host (one emulated CTA of 1024
    threads, every array its own exactly sized heap buffer under
    AddressSanitizer) against its rules written out in the test: the one-pass
    form (capacity and cells at most 1024), a first frame, lists truncated at
    the capacity, and the multi-pass form (2000 slots, 1980 cells)."""
    W, H, cw, ch, k = {"one_pass": (376, 240, 40, 40, 2), "first_frame": (376, 240, 40, 40, 2),
                       "truncated": (376, 240, 40, 40, 3),
                       "multi_pass": (1920, 1080, 32, 32, 1)}[case]
    cells = (W // cw) * (H // ch)
    cap = {"one_pass": 216, "first_frame": 216, "truncated": 120, "multi_pass": 2000}[case]
    rng = np.random.default_rng({"one_pass": 1, "first_frame": 2, "truncated": 3,
                                 "multi_pass": 4}[case])
    n0, n1 = int(cap * 0.7), int(cap * 0.55)
    if case == "truncated":
        n0, n1 = cap - 3, cap - 10
    have_prev = 0 if case == "first_frame" else 1
    trk_status = np.where(rng.random(2 * cap) < 0.75, 0, rng.integers(1, 7, 2 * cap)).astype(
        np.uint8)
    trk_xy = np.stack([rng.uniform(-2, W + 2, 2 * cap), rng.uniform(-2, H + 2, 2 * cap)],
                      1).astype(np.float32)
    trk_xy[:8] = [[0, 0], [cw, ch], [cw - 1e-4, 0], [W - 1, H - 1], [-0.5, 3], [W - 0.001, 5],
                  [(W // cw) * cw, 7], [3, (H // ch) * ch]]
    # every cell edge and the float just below it, in x and in y (the cell of
    # a position must be exact where x / cw rounds onto an integer)
    edges = np.arange(1, W // cw + 1, dtype=np.float32) * np.float32(cw)
    ex = np.concatenate([edges, np.nextafter(edges, np.float32(0))])
    edges = np.arange(1, H // ch + 1, dtype=np.float32) * np.float32(ch)
    ey = np.concatenate([edges, np.nextafter(edges, np.float32(0))])
    m = min(len(ex), (n0 - 8) // 2)
    trk_xy[8:8 + m, 0] = ex[:m]
    m2 = min(len(ey), n0 - 8 - m)
    trk_xy[8 + m:8 + m + m2, 1] = ey[:m2]
    trk_status[:8 + m + m2] = 0
    if case == "truncated":
        trk_xy[:cap, 0] = -1.0     # camera-0 survivors outside the grid: no occupancy
    list_id = rng.integers(0, 1 << 20, 2 * cap).astype(np.int32)
    cand_count = rng.integers(0, k + 1, cells).astype(np.int32)
    if case == "truncated":
        cand_count[:] = k          # more new keypoints than the capacity
    idx = rng.integers(0, W * H, cells * k).astype(np.uint64)
    score = rng.integers(1, 255, cells * k).astype(np.uint64)
    cand = ((score << np.uint64(32)) | (~idx & np.uint64(0xffffffff))).astype(np.uint64)
    spec_status = np.where(rng.random(cells * k) < 0.8, 0, 5).astype(np.uint8)
    spec_xy = rng.uniform(0, W, (cells * k, 2)).astype(np.float32)
    next_id = 1000
    inp, outp = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        f.write(np.array([W, H, cw, ch, k, cap, n0, n1, next_id, have_prev], np.int32).tobytes())
        for a in (trk_status, trk_xy, list_id, cand_count, cand, spec_status, spec_xy):
            f.write(np.ascontiguousarray(a).tobytes())
    _run(_build(tmp_path, "fin_check"), inp, outp, timeout=900, expect="finalised")
    b = open(outp, "rb").read()
    o = 0

    def take(dt, n):
        nonlocal o
        a = np.frombuffer(b, dt, n, o)
        o += a.nbytes
        return a
    cnt = take(np.int32, 2)
    lxy = take(np.float32, 4 * cap).reshape(2, cap, 2)
    lid = take(np.int32, 2 * cap).reshape(2, cap)
    lst = take(np.uint8, 2 * cap).reshape(2, cap)
    new_count = int(take(np.int32, 1)[0])
    new_xy = take(np.float32, 2 * cap).reshape(cap, 2)
    nid = int(take(np.int32, 1)[0])
    occ = take(np.uint8, cells)
    stats = take(np.int32, 8)
    e = _finalize_expected(W, H, cw, ch, k, cap, n0, n1, next_id, have_prev, trk_status,
                           trk_xy, list_id, cand_count, cand, spec_status, spec_xy)
    assert cnt.tolist() == e["count"]
    for c in range(2):
        n = e["count"][c]
        assert np.array_equal(lxy[c, :n], np.array(e["xy"][c], np.float32).reshape(-1, 2)), c
        assert np.array_equal(lid[c, :n], np.array(e["id"][c], np.int32)), c
        assert np.all(lst[c, :n] == 0) and np.all(lst[c, n:] == 255), c
    assert new_count == e["new_count"] and nid == e["next_id"]
    assert np.array_equal(new_xy[:new_count], np.array(e["new_xy"], np.float32).reshape(-1, 2))
    assert np.array_equal(occ, e["occ"].astype(np.uint8))
    assert stats.tolist() == e["stats"]
    if case == "truncated":
        assert e["count"][0] == cap and e["stats"][4] > cap


@pytest.mark.parametrize("radius", [1.0, 3.0])
def test_initnet_training_pass_on_host(tmp_path, radius):
    """The flow network's training pass (per-warp forward on mma.sync tiles,
    the loss, the FP32 backward, the gradient sums) on the host, its shared
    memory exactly train_smem_bytes() under AddressSanitizer, against the
    FP64 oracle's batch gradient at the GPU test's per-element bound; 14
    samples over 4 warps, so warps take several samples and share the
    accumulator."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from initnet_util import GRAD_REL, KINK_MARGIN, _abs_grad, _kink_margin
    rng = np.random.default_rng(11 + int(radius))
    fan = {"w1": 36, "w2": 288, "w3": 288, "w4": 128, "w5": 64}
    p = {k: (rng.normal(0, np.sqrt(2.0 / fan[k]), onet.SHAPES[k]) if k.startswith("w")
             else rng.normal(0, 0.05, onet.SHAPES[k])) for k in onet.ORDER}
    p = onet.unflatten(onet.flatten(p).astype(np.float32).astype(np.float64))
    pb = {k: (onet.bf16_round(v) if k.startswith("w") else v) for k, v in p.items()}
    n = 14
    xs = []
    while len(xs) < n:
        xi = (rng.integers(0, 256, (4, 16, 16)).astype(np.float64) - 128) / 64
        if _kink_margin(pb, xi) > KINK_MARGIN:
            xs.append(xi)
    x = np.stack(xs)
    flows = []
    for xi in x:
        o = onet.forward(pb, xi, act_bf16=True)
        r = rng.choice([rng.uniform(0.0, 0.8 * radius), rng.uniform(1.2 * radius, 6.0 * radius)])
        a = rng.uniform(0, 2 * np.pi)
        flows.append([o[0] * 16 + r * np.cos(a), o[1] * 16 + r * np.sin(a)])
    flows = np.array(flows, np.float32).astype(np.float64)
    loss_ref, g_ref = onet.batch_loss_grad(pb, x, flows, act_bf16=True, radius=radius)
    g_abs = _abs_grad(pb, x, flows, radius)
    xb = (x.reshape(n, -1).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    inp, outp = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        f.write(np.array([n], np.int32).tobytes())
        f.write(np.array([1.0 / n, radius], np.float32).tobytes())
        f.write(_packed(p))
        f.write(xb.tobytes())
        f.write(flows.astype(np.float32).tobytes())
    _run(_build(tmp_path, "train_check"), inp, outp, timeout=1200, expect="trained")
    out = np.fromfile(outp, np.float32)
    grad, loss = out[:-1].astype(np.float64), float(out[-1])
    assert loss / n == pytest.approx(loss_ref, rel=1e-3)
    g = onet.unflatten(grad)
    for k in onet.ORDER:
        bound = GRAD_REL * g_abs[k] + 1e-7 * np.abs(g_abs[k]).max()
        err = np.abs(g[k] - g_ref[k])
        assert np.all(err <= bound), (k, float((err / np.maximum(bound, 1e-300)).max()))
        assert np.median(err / np.maximum(g_abs[k], 1e-300)) < 1e-4, k


@pytest.mark.parametrize("la,lb", [(2, 3), (1, 2)])
def test_network_input_extraction_on_host(tmp_path, la, lb):
    """The flow network's input, both device forms (the warp's extraction and
    the frame launch's aligned-word prefetch with its per-byte BF16
    conversion), read from levels between poisoned gaps with padded pitches
    full of other bytes, bit for bit against the oracle's extraction:
    interior keypoints, keypoints at and past the borders, positions on the
    rounding half."""
    from paper_2609_30459_gb300 import synth
    oracle.build()
    w, h, L = 218, 151, 4
    seq = synth.make_sequence(7200, 2, w, h, 1, max_motion=6.0, tex_size=1024)
    src = oracle.pyramid(seq.frames[0, 0], L)
    dst = oracle.pyramid(seq.frames[1, 0], L)
    rng = np.random.default_rng(la * 10 + lb)
    pts = np.concatenate([
        np.stack([rng.uniform(0, w, 20), rng.uniform(0, h, 20)], 1),
        np.array([[0, 0], [w - 1, h - 1], [2, 75], [w - 3, 75], [100, 1], [100, h - 2],
                  [-6, 40], [w + 5, 40], [40, -9], [40, h + 7], [12.0, 20.0], [14.0, 22.0],
                  [63.999, 17.5], [64.0, 18.0]])]).astype(np.float32)
    inp, outp = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        f.write(np.array([L, len(pts), la, lb], np.int32).tobytes())
        for l in range(L):
            f.write(np.array(src[l].shape[::-1], np.int32).tobytes())
            f.write(np.ascontiguousarray(src[l], np.uint8).tobytes())
            f.write(np.ascontiguousarray(dst[l], np.uint8).tobytes())
        f.write(pts.tobytes())
    _run(_build(tmp_path, "netin_check"), inp, outp, timeout=600, expect="inputs")
    got = np.fromfile(outp, np.uint16).reshape(len(pts), 2, 4, 16, 16)
    for i, (x, y) in enumerate(pts):
        ref = onet.extract(src, dst, float(x), float(y), la, lb)
        bits = _bf16_bits(ref)
        assert np.array_equal(got[i, 0], bits), ("warp", i, x, y)
        assert np.array_equal(got[i, 1], bits), ("prefetch", i, x, y)
