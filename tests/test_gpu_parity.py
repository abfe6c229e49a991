"""GPU parity: every stage through the C ABI against the CPU oracle on the
same seeded inputs. Bit-exact for the pyramid, FAST scores and detection;
flow within 1e-3 px and explained status disagreements for tracking."""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_30459_gb300 import synth
from tests.parity_util import compare_tracks

pytestmark = pytest.mark.gpu

vio = pytest.importorskip("paper_2609_30459_gb300.vio")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vio.load(build=True)
    oracle.build()


DEV = "cuda"


def textured(seed, h, w, sigma=2.0, noise=2.0):
    rng = np.random.default_rng(seed)
    return synth.quantize(synth.band_limited_texture(seed, h, w, sigma), rng, noise)


def to_dev(imgs, pitch=None):
    """(n, h, w) uint8 numpy -> (n, h, pitch) CUDA tensor (padding = 0)."""
    n, h, w = imgs.shape
    pitch = pitch or w
    t = torch.zeros((n, h, pitch), dtype=torch.uint8)
    t[:, :, :w] = torch.from_numpy(imgs)
    return t.to(DEV)


# ---------------------------------------------------------------- pyramid ---

@pytest.mark.parametrize("w,h,L", [(752, 480, 4), (1920, 1080, 5), (131, 77, 3), (640, 480, 4),
                                   (1280, 720, 5), (33, 17, 2), (5, 4, 3), (1, 1, 1)])
@pytest.mark.parametrize("mode", [0, 1])
def test_pyramid_bitexact(w, h, L, mode):
    imgs = np.stack([textured(100 + i, h, w) for i in range(3)])
    imgs[2, : h // 2, : w // 3] = 255                     # saturated block
    pitch = w + (13 if w > 8 else 0)                      # ragged pitch
    pyr = vio.Pyramids(to_dev(imgs, pitch), L, w=w)
    ctx = vio.Context(vio.default_params(n_levels=L, round_mode=mode), w, h, 3)
    ctx.pyramid_build(pyr)
    torch.cuda.synchronize()
    for i in range(3):
        ref = oracle.pyramid(imgs[i], L, mode)
        for l in range(1, L):
            assert np.array_equal(pyr.level(i, l).cpu().numpy(), ref[l]), (i, l)


# ------------------------------------------------------------------- FAST ---

@pytest.mark.parametrize("w,h", [(752, 480), (1920, 1080), (97, 41), (7, 7), (6, 9)])
def test_fast_scores_bitexact(w, h):
    img = textured(7, h, w, sigma=1.2, noise=4.0)
    if h > 20 and w > 20:
        img[10:15, 10:15] = 255
        img[5, :] = 0
    t = to_dev(img[None], w + 3)[0]
    got = vio.fast_scores(t, w=w)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), oracle.fast_scores(img))


# -------------------------------------------------------------- detection ---

DETECT_CASES = [
    # w, h, cell_w, cell_h, k, thresholds, border
    (752, 480, 94, 60, 2, (40, 20, 10, 5), 9),      # 8x8 grid, k = 2
    (752, 480, 50, 50, 1, (40, 20, 10, 5), 9),      # paper default cell
    (752, 480, 37, 32, 1, (40, 20, 10, 5), 9),      # 20x15 grid
    (1920, 1080, 48, 43, 1, (40, 20, 10, 5), 9),    # 40x25 grid
    (640, 480, 82, 82, 1, (40, 20), 9),             # lite: min threshold 20, cell 82
    (300, 200, 30, 25, 8, (40, 20, 10, 5), 3),      # k = 8, small border
    (257, 131, 16, 16, 3, (10,), 0),                # ragged cells, no border
]


@pytest.mark.parametrize("w,h,cw,ch,k,thr,border", DETECT_CASES)
def test_detect_bitexact(w, h, cw, ch, k, thr, border):
    n = 3
    imgs = np.stack([textured(200 + i, h, w, sigma=1.5) for i in range(n)])
    gx, gy = w // cw, h // ch
    rng = np.random.default_rng(w + k)
    occ = rng.integers(0, k + 1, (n, gx * gy)).astype(np.uint8)
    occ[0] = 0
    mask = (rng.random((n, h, w)) > 0.05).astype(np.uint8)
    mask[0] = 1
    p = vio.default_params(n_levels=1, cell_w=cw, cell_h=ch, k_per_cell=k, thresholds=thr,
                           detect_border=border)
    ctx = vio.Context(p, w, h, n)
    pyr = vio.Pyramids(to_dev(imgs), 1)
    cap = gx * gy * k
    kp = torch.full((n, max(cap, 1), 2), -1.0, device=DEV)
    sc = torch.zeros((n, max(cap, 1)), dtype=torch.int16, device=DEV)
    cnt = torch.zeros(n, dtype=torch.int32, device=DEV)
    d_occ = torch.from_numpy(occ).to(DEV)
    d_mask = torch.from_numpy(mask).to(DEV)
    ctx.detect_grid(pyr, pyr.batch(), kp, sc, cnt, cap, occupancy=d_occ, mask=d_mask,
                    mask_stride=h * w)
    torch.cuda.synchronize()
    for i in range(n):
        rk, rs = oracle.detect_grid(imgs[i], cw, ch, k=k, thresholds=thr, border=border,
                                    occupancy=occ[i], mask=mask[i])
        c = int(cnt[i])
        assert c == len(rk), (i, c, len(rk))
        assert np.array_equal(kp[i, :c].cpu().numpy(), rk)
        assert np.array_equal(sc[i, :c].cpu().numpy(), rs)


@pytest.mark.parametrize("masked", [False, True])
def test_detect_many_large_cells_bitexact(masked):
    """A batch with enough cells that each gets a single warp, with large
    cells and the full threshold sequence: a warp scores more pixels than its
    queue holds, so candidates come from the scan of its part of the map.
    Every image bit-exact against the oracle."""
    n, w, h, cw, ch, k, thr = 56, 752, 480, 82, 82, 2, (40, 20, 10, 5)
    imgs = np.stack([textured(900 + i, h, w, sigma=1.2, noise=3.0) for i in range(n)])
    gx, gy = w // cw, h // ch
    mask = None
    if masked:
        mask = (np.random.default_rng(7).random((n, h, w)) > 0.1).astype(np.uint8)
    p = vio.default_params(n_levels=1, cell_w=cw, cell_h=ch, k_per_cell=k, thresholds=thr,
                           detect_border=9)
    ctx = vio.Context(p, w, h, n)
    pyr = vio.Pyramids(to_dev(imgs), 1)
    cap = gx * gy * k
    kp = torch.full((n, cap, 2), -1.0, device=DEV)
    sc = torch.zeros((n, cap), dtype=torch.int16, device=DEV)
    cnt = torch.zeros(n, dtype=torch.int32, device=DEV)
    if masked:
        ctx.detect_grid(pyr, pyr.batch(), kp, sc, cnt, cap,
                        mask=torch.from_numpy(mask).to(DEV), mask_stride=h * w)
    else:
        ctx.detect_grid(pyr, pyr.batch(), kp, sc, cnt, cap)
    torch.cuda.synchronize()
    for i in range(n):
        rk, rs = oracle.detect_grid(imgs[i], cw, ch, k=k, thresholds=thr, border=9,
                                    mask=mask[i] if masked else None)
        c = int(cnt[i])
        assert c == len(rk), (i, c, len(rk))
        assert np.array_equal(kp[i, :c].cpu().numpy(), rk)
        assert np.array_equal(sc[i, :c].cpu().numpy(), rs)


# The paper's three per-cell selections (Sec. III-D: k rounds of a maximum,
# a bitonic k-sort, an atomic maximum for one keypoint per cell) pick the same
# keys (unique under the (score, y, x) order), so each must match the oracle
# bit for bit, through the standalone detection and the fused pyramid launch.
@pytest.mark.parametrize("k,mode", [(1, 0), (1, 1), (1, 2), (2, 0), (2, 1), (8, 0), (8, 1)])
@pytest.mark.parametrize("fused", [False, True])
def test_detect_selection_modes_bitexact(k, mode, fused):
    n, w, h, cw, ch = 4, 640, 400, 40, 32
    imgs = np.stack([textured(300 + i, h, w, sigma=1.5) for i in range(n)])
    gx, gy = w // cw, h // ch
    occ = np.random.default_rng(k + 10 * mode).integers(0, k + 1, (n, gx * gy)).astype(np.uint8)
    occ[0] = 0
    p = vio.default_params(n_levels=3, cell_w=cw, cell_h=ch, k_per_cell=k, select_mode=mode)
    ctx = vio.Context(p, w, h, n)
    pyr = vio.Pyramids(to_dev(imgs), 3)
    cap = gx * gy * k
    kp = torch.full((n, cap, 2), -1.0, device=DEV)
    sc = torch.zeros((n, cap), dtype=torch.int16, device=DEV)
    cnt = torch.zeros(n, dtype=torch.int32, device=DEV)
    d_occ = torch.from_numpy(occ).to(DEV)
    if fused:
        ctx.pyramid_detect(pyr, kp, sc, cnt, cap, occupancy=d_occ)
    else:
        ctx.detect_grid(pyr, pyr.batch(), kp, sc, cnt, cap, occupancy=d_occ)
    torch.cuda.synchronize()
    for i in range(n):
        rk, rs = oracle.detect_grid(imgs[i], cw, ch, k=k, border=p.detect_border,
                                    occupancy=occ[i])
        c = int(cnt[i])
        assert c == len(rk), (i, c, len(rk))
        assert np.array_equal(kp[i, :c].cpu().numpy(), rk)
        assert np.array_equal(sc[i, :c].cpu().numpy(), rs)
    ctx.close()


def test_detect_atomic_selection_needs_k1():
    p = vio.default_params(n_levels=1, cell_w=40, cell_h=40, k_per_cell=2, select_mode=2)
    with pytest.raises(vio.VioError):
        vio.Context(p, 160, 120, 1)
    p = vio.default_params(n_levels=1, cell_w=40, cell_h=40, k_per_cell=1, select_mode=3)
    with pytest.raises(vio.VioError):
        vio.Context(p, 160, 120, 1)


def test_detect_capacity_truncates_in_raster_order():
    w, h = 400, 300
    img = textured(5, h, w)
    p = vio.default_params(n_levels=1, cell_w=40, cell_h=30, k_per_cell=2)
    ctx = vio.Context(p, w, h, 1)
    pyr = vio.Pyramids(to_dev(img[None]), 1)
    cap = 37
    kp = torch.zeros((1, cap, 2), device=DEV)
    sc = torch.zeros((1, cap), dtype=torch.int16, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int32, device=DEV)
    ctx.detect_grid(pyr, pyr.batch(), kp, sc, cnt, cap)
    rk, rs = oracle.detect_grid(img, 40, 30, k=2, border=p.detect_border, capacity=cap)
    torch.cuda.synchronize()
    assert int(cnt[0]) == len(rk) == cap
    assert np.array_equal(kp[0].cpu().numpy(), rk) and np.array_equal(sc[0].cpu().numpy(), rs)


def test_detect_flat_image_finds_nothing():
    img = np.full((1, 120, 160), 77, np.uint8)
    p = vio.default_params(n_levels=1, cell_w=40, cell_h=40)
    ctx = vio.Context(p, 160, 120, 1)
    pyr = vio.Pyramids(to_dev(img), 1)
    kp = torch.zeros((1, 12, 2), device=DEV)
    sc = torch.zeros((1, 12), dtype=torch.int16, device=DEV)
    cnt = torch.full((1,), -5, dtype=torch.int32, device=DEV)
    ctx.detect_grid(pyr, pyr.batch(), kp, sc, cnt, 12)
    torch.cuda.synchronize()
    assert int(cnt[0]) == 0


# --------------------------------------------------------------- tracking ---

def _pair_case(seed, w, h, L, n_pts, max_t=3.0):
    d = synth.stereo_pair_small_motion(seed, w, h, max_t=max_t)
    imgs = d["images"]
    kp, _ = oracle.detect_grid(imgs[0, 0], max(w // 20, 12), max(h // 15, 12), k=1, border=9)
    kp = kp[:n_pts]
    return imgs, kp


@pytest.mark.parametrize("w,h,L,n", [(752, 480, 3, 150), (752, 480, 4, 300),
                                     (1920, 1080, 5, 1000), (200, 150, 3, 40)])
@pytest.mark.parametrize("fb", [True, False])
def test_track_temporal_parity(w, h, L, n, fb):
    imgs, kp = _pair_case(31 + L, w, h, L, n)
    p = vio.default_params(n_levels=L)
    ctx = vio.Context(p, w, h, 4)
    pyr = vio.Pyramids(to_dev(imgs.reshape(4, h, w)), L)
    ctx.pyramid_build(pyr)
    cap = len(kp) + 7                                       # ragged tail of empty slots
    pts = torch.zeros((1, cap, 2), device=DEV)
    pts[0, : len(kp)] = torch.from_numpy(kp)
    cnt = torch.tensor([len(kp)], dtype=torch.int32, device=DEV)
    out = torch.zeros((1, cap, 3), device=DEV)
    st = torch.zeros((1, cap), dtype=torch.uint8, device=DEV)
    fbd = torch.zeros((1, cap), device=DEV)
    ls = torch.zeros((1, cap), device=DEV)
    for cam in (0, 1):
        ctx.track_patches(pyr, pyr.batch(cam, 1, 1), pyr.batch(2 + cam, 1, 1), pts, cnt, cap,
                          out, st, fbd, fb=fb, last_step=ls)
        torch.cuda.synchronize()
        ref = oracle.track(oracle.pyramid(imgs[0, cam], L), oracle.pyramid(imgs[1, cam], L), kp,
                           fb=fb, fb_max_dist=p.fb_max_dist, n_threads=8)
        s = compare_tracks(out[0, : len(kp), :2].cpu().numpy(), st[0, : len(kp)].cpu().numpy(),
                           ref, p.fb_max_dist, g_theta=out[0, : len(kp), 2].cpu().numpy())
        assert s["n_ok"] >= 0.5 * len(kp), s
        assert (st[0, len(kp):] == 255).all()
        both = (st[0, : len(kp)].cpu().numpy() == 0) & (ref["status"] == 0)
        if fb:
            dd = np.abs(fbd[0, : len(kp)].cpu().numpy()[both] - ref["fb_dist"][both])
            assert dd.max() < 1e-3
        # the convergence measure (the learned start's gate): the last level-0
        # step, |dx| + |dy| + r |dth|, to 1e-4 px plus 1% where it is large
        gl = ls[0, : len(kp)].cpu().numpy().astype(np.float64)[both]
        assert np.all(np.abs(gl - ref["last_step"][both]) <= 1e-4 + 0.01 * ref["last_step"][both])


def test_track_with_init_and_empty():
    w, h, L = 320, 240, 3
    imgs, kp = _pair_case(77, w, h, L, 60)
    p = vio.default_params(n_levels=L)
    ctx = vio.Context(p, w, h, 4)
    pyr = vio.Pyramids(to_dev(imgs.reshape(4, h, w)), L)
    ctx.pyramid_build(pyr)
    rng = np.random.default_rng(0)
    init = np.concatenate([kp + rng.uniform(-1, 1, kp.shape).astype(np.float32),
                           rng.uniform(-0.01, 0.01, (len(kp), 1)).astype(np.float32)], 1)
    cap = len(kp)
    pts = torch.from_numpy(kp).to(DEV)[None]
    d_init = torch.from_numpy(init).to(DEV)[None]
    cnt = torch.tensor([cap], dtype=torch.int32, device=DEV)
    out = torch.zeros((1, cap, 3), device=DEV)
    st = torch.zeros((1, cap), dtype=torch.uint8, device=DEV)
    ctx.track_patches(pyr, pyr.batch(0, 1, 1), pyr.batch(2, 1, 1), pts, cnt, cap, out, st,
                      init=d_init)
    torch.cuda.synchronize()
    ref = oracle.track(oracle.pyramid(imgs[0, 0], L), oracle.pyramid(imgs[1, 0], L), kp,
                       init=init, fb_max_dist=p.fb_max_dist)
    compare_tracks(out[0, :, :2].cpu().numpy(), st[0].cpu().numpy(), ref, p.fb_max_dist,
                   g_theta=out[0, :, 2].cpu().numpy())
    # zero keypoints: every slot EMPTY, nothing else touched
    cnt.zero_()
    ctx.track_patches(pyr, pyr.batch(0, 1, 1), pyr.batch(2, 1, 1), pts, cnt, cap, out, st)
    torch.cuda.synchronize()
    assert (st == 255).all()


@pytest.mark.parametrize("w,h,L,n", [(752, 480, 4, 300), (1920, 1080, 5, 1000)])
def test_stereo_match_parity(w, h, L, n):
    imgs, kp = _pair_case(55 + L, w, h, L, n)
    p = vio.default_params(n_levels=L)
    ctx = vio.Context(p, w, h, 2)
    pyr = vio.Pyramids(to_dev(imgs[0]), L)                  # cam0, cam1 at time t
    ctx.pyramid_build(pyr)
    cap = len(kp)
    pts = torch.from_numpy(kp).to(DEV)[None]
    cnt = torch.tensor([cap], dtype=torch.int32, device=DEV)
    m = torch.zeros((1, cap, 2), device=DEV)
    st = torch.zeros((1, cap), dtype=torch.uint8, device=DEV)
    ctx.stereo_match(pyr, pyr.batch(0, 1, 1), pyr.batch(1, 1, 1), pts, cnt, cap, m, st)
    torch.cuda.synchronize()
    ref = oracle.track(oracle.pyramid(imgs[0, 0], L), oracle.pyramid(imgs[0, 1], L), kp,
                       fb_max_dist=p.fb_max_dist, n_threads=8)
    s = compare_tracks(m[0].cpu().numpy(), st[0].cpu().numpy(), ref, p.fb_max_dist)
    assert s["n_ok"] >= 0.3 * cap, s


def test_fb_check_kernel():
    rng = np.random.default_rng(3)
    n_img, cap = 2, 50
    orig = rng.uniform(0, 100, (n_img, cap, 2)).astype(np.float32)
    back = np.concatenate([orig + rng.normal(0, 0.2, orig.shape).astype(np.float32),
                           np.zeros((n_img, cap, 1), np.float32)], 2)
    status = rng.choice([0, 0, 0, 2], (n_img, cap)).astype(np.uint8)
    cnt = np.array([cap, 31], np.int32)
    d_st = torch.from_numpy(status).to(DEV)
    d_dist = torch.full((n_img, cap), -1.0, device=DEV)
    vio.fb_check(torch.from_numpy(orig).to(DEV), torch.from_numpy(back).to(DEV),
                 torch.from_numpy(cnt).to(DEV), cap, n_img, 0.25, d_st, d_dist)
    torch.cuda.synchronize()
    dist = np.hypot(*(back[..., :2] - orig).transpose(2, 0, 1))
    exp = status.copy()
    for i in range(n_img):
        for k in range(cnt[i]):
            if status[i, k] == 0 and not dist[i, k] <= 0.25:
                exp[i, k] = 5
    assert np.array_equal(d_st.cpu().numpy(), exp)
    got = d_dist.cpu().numpy()
    live = (status == 0) & (np.arange(cap)[None] < cnt[:, None])
    assert np.allclose(got[live], dist[live], atol=1e-5)
    assert (got[~live] == -1).all()


@pytest.mark.parametrize("w,h,L,cw,ch,k", [(752, 480, 4, 37, 32, 1), (1920, 1080, 5, 48, 43, 1),
                                           (640, 480, 6, 50, 50, 2), (300, 200, 2, 30, 25, 3),
                                           (131, 77, 1, 20, 16, 1)])
def test_pyramid_detect_fused_bitexact(w, h, L, cw, ch, k):
    n = 3
    imgs = np.stack([textured(300 + i, h, w, sigma=1.5) for i in range(n)])
    gx, gy = w // cw, h // ch
    rng = np.random.default_rng(w + L)
    occ = rng.integers(0, k + 1, (n, gx * gy)).astype(np.uint8)
    mask = (rng.random((n, h, w)) > 0.05).astype(np.uint8)
    p = vio.default_params(n_levels=L, cell_w=cw, cell_h=ch, k_per_cell=k)
    ctx = vio.Context(p, w, h, n)
    pyr = vio.Pyramids(to_dev(imgs, w + 32), L, w=w)
    cap = gx * gy * k
    kp = torch.zeros((n, cap, 2), device=DEV)
    sc = torch.zeros((n, cap), dtype=torch.int16, device=DEV)
    cnt = torch.zeros(n, dtype=torch.int32, device=DEV)
    ctx.pyramid_detect(pyr, kp, sc, cnt, cap, occupancy=torch.from_numpy(occ).to(DEV),
                       mask=torch.from_numpy(mask).to(DEV), mask_stride=h * w)
    torch.cuda.synchronize()
    for i in range(n):
        ref = oracle.pyramid(imgs[i], L)
        for l in range(1, L):
            assert np.array_equal(pyr.level(i, l).cpu().numpy(), ref[l]), (i, l)
        rk, rs = oracle.detect_grid(imgs[i], cw, ch, k=k, border=p.detect_border,
                                    occupancy=occ[i], mask=mask[i])
        c = int(cnt[i])
        assert c == len(rk)
        assert np.array_equal(kp[i, :c].cpu().numpy(), rk)
        assert np.array_equal(sc[i, :c].cpu().numpy(), rs)


def test_detect_low_contrast_falls_back_to_all_thresholds():
    # weak texture: most cells only reach the smaller thresholds, so the
    # bound-driven search must go down to T_min
    w, h = 400, 300
    img = synth.quantize(128 + 0.08 * (synth.band_limited_texture(9, h, w, 2.0) - 128),
                         np.random.default_rng(1), 1.0)
    p = vio.default_params(n_levels=1, cell_w=40, cell_h=30, k_per_cell=3)
    ctx = vio.Context(p, w, h, 1)
    pyr = vio.Pyramids(to_dev(img[None]), 1)
    cap = 10 * 10 * 3
    kp = torch.zeros((1, cap, 2), device=DEV)
    sc = torch.zeros((1, cap), dtype=torch.int16, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int32, device=DEV)
    ctx.detect_grid(pyr, pyr.batch(), kp, sc, cnt, cap)
    torch.cuda.synchronize()
    rk, rs = oracle.detect_grid(img, 40, 30, k=3, border=p.detect_border)
    c = int(cnt[0])
    assert c == len(rk) and c > 0 and rs.min() < 20
    assert np.array_equal(kp[0, :c].cpu().numpy(), rk) and np.array_equal(sc[0, :c].cpu().numpy(), rs)
