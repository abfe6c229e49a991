"""Pins of the CPU oracle's pyramid and detector against what the paper and
the mathematics fix (Sec. III-C, Eq. 1-3; Sec. III-D). No GPU."""
import itertools
import json
import os

import numpy as np
import pytest
from scipy import ndimage

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")
W5 = np.array([1, 4, 6, 4, 1])


@pytest.fixture(scope="module")
def consts():
    with open(GOLDEN) as f:
        return json.load(f)


def rnd(seed, h, w, lo=0, hi=256):
    return np.random.default_rng(seed).integers(lo, hi, (h, w)).astype(np.uint8)


# ---------------------------------------------------------------- pyramid ---

@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("c", [0, 1, 77, 255])
def test_pyramid_constant_image(mode, c):
    img = np.full((37, 53), c, np.uint8)
    for lv in oracle.pyramid(img, 4, mode)[1:]:
        assert np.all(lv == c)


def test_pyramid_level_sizes_floor():
    lv = oracle.pyramid(np.zeros((1080, 1920), np.uint8), 5)
    assert [a.shape for a in lv] == [(1080, 1920), (540, 960), (270, 480), (135, 240), (67, 120)]


@pytest.mark.parametrize("mode", [0, 1])
def test_pyramid_linear_ramp_interior_is_subsampling(mode):
    # The binomial kernel is symmetric with sum 256, so a linear ramp is
    # reproduced exactly at the tap centre 2x, 2y away from the clamped border.
    h, w = 48, 64
    y, x = np.mgrid[0:h, 0:w]
    img = (1 * x + 2 * y + 20).astype(np.uint8)
    l1 = oracle.pyr_down(img, mode)
    assert np.array_equal(l1[1:-1, 1:-1], img[2:-2:2, 2:-2:2][: h // 2 - 2, : w // 2 - 2])


@pytest.mark.parametrize("mode,expect", [(0, {0: 36, 1: 6, 2: 1}), (1, {0: 35, 1: 5, 2: 0})])
def test_pyramid_impulse_even(mode, expect):
    # 255 at (2X, 2Y): L1(X+dx, Y+dy) = round(255 * w_{2dx} w_{2dy} / 256):
    # centre 255*36/256 = 35.86, edge 255*6/256 = 5.98, corner 255/256.
    img = np.zeros((32, 32), np.uint8)
    img[12, 16] = 255
    l1 = oracle.pyr_down(img, mode).astype(int)
    X, Y = 8, 6
    assert l1[Y, X] == expect[0]
    for dx, dy in [(1, 0), (-1, 0), (0, 1), (0, -1)]:
        assert l1[Y + dy, X + dx] == expect[1]
    for dx, dy in [(1, 1), (-1, 1), (1, -1), (-1, -1)]:
        assert l1[Y + dy, X + dx] == expect[2]
    l1[Y - 1:Y + 2, X - 1:X + 2] = 0
    assert not l1.any()


def test_pyramid_impulse_odd():
    # 255 at (2X+1, 2Y): taps i = +1 (from X) and i = -1 (from X+1), weight 4.
    img = np.zeros((32, 32), np.uint8)
    img[12, 17] = 255
    l1 = oracle.pyr_down(img, 0).astype(int)
    assert l1[6, 8] == l1[6, 9] == round(255 * 4 * 6 / 256)      # 23.9 -> 24
    assert l1[5, 8] == l1[7, 9] == round(255 * 4 * 1 / 256)      # 3.98 -> 4


@pytest.mark.parametrize("shape", [(31, 45), (48, 64), (17, 9)])
@pytest.mark.parametrize("mode", [0, 1])
def test_pyramid_matches_library_correlation(shape, mode):
    # scipy's correlation with the 5x5 outer-product kernel and edge
    # replication ('nearest'), sampled at even positions, then rounded.
    img = rnd(sum(shape) + mode, *shape)
    k = np.outer(W5, W5)
    s = ndimage.correlate(img.astype(np.int64), k, mode="nearest")
    s = s[0:2 * (shape[0] // 2):2, 0:2 * (shape[1] // 2):2]
    ref = (s + 128) >> 8 if mode == 0 else s >> 8
    assert np.array_equal(oracle.pyr_down(img, mode), ref.astype(np.uint8))


@pytest.mark.parametrize("mode", [0, 1])
def test_pyramid_separable_form_equals_double_sum(mode):
    # Eq. 2-3 (horizontal pass at stride 2, then vertical, then the shift)
    # must agree with Eq. 1's double sum bit for bit.
    img = rnd(5, 41, 58).astype(np.int64)
    h, w = img.shape
    xs = np.clip(2 * np.arange(w // 2)[:, None] + np.arange(-2, 3)[None, :], 0, w - 1)
    V = (img[:, xs] * W5[None, None, :]).sum(-1)                     # (h, w/2)
    ys = np.clip(2 * np.arange(h // 2)[:, None] + np.arange(-2, 3)[None, :], 0, h - 1)
    S = (V[ys, :] * W5[None, :, None]).sum(1)                         # (h/2, w/2)
    ref = (S + 128) >> 8 if mode == 0 else S >> 8
    assert np.array_equal(oracle.pyr_down(img.astype(np.uint8), mode), ref)


def test_pyramid_tile_footprint_within_paper_region(consts):
    # Sec. III-C: a 32x8 output tile reads a (2S+4)x(2R+4) = 68x20 region.
    # Measure the oracle's footprint by perturbing one source pixel at a time.
    t = consts["pyramid_tile"]
    S, R = t["S"], t["R"]
    base = rnd(1, 40, 80)
    ref = oracle.pyr_down(base, 1).astype(int)
    xs, ys = set(), set()
    for y in range(40):
        for x in range(80):
            b = base.copy()
            b[y, x] = 255 - b[y, x]
            d = oracle.pyr_down(b, 1).astype(int) != ref
            # does any pixel of the output tile [4, 4+S) x [4, 4+R) change?
            if d[4:4 + R, 4:4 + S].any():
                xs.add(x)
                ys.add(y)
    fw, fh = max(xs) - min(xs) + 1, max(ys) - min(ys) + 1
    assert (fw, fh) == (2 * S + 3, 2 * R + 3)
    assert fw <= t["source_region"][0] and fh <= t["source_region"][1]


# ------------------------------------------------------------------- FAST ---

def midpoint_circle(r):
    """Bresenham's midpoint circle, all octants, as a set of offsets."""
    pts = set()
    x, y, d = r, 0, 1 - r
    while x >= y:
        for sx, sy in itertools.product((1, -1), repeat=2):
            pts.add((sx * x, sy * y))
            pts.add((sx * y, sy * x))
        y += 1
        if d < 0:
            d += 2 * y + 1
        else:
            x -= 1
            d += 2 * (y - x) + 1
    return pts


def test_fast_ring_geometry(consts):
    dx, dy = oracle.fast_ring()
    ring = list(zip(dx.tolist(), dy.tolist()))
    assert len(ring) == consts["fast_ring_points"]["value"] == 16
    assert set(ring) == midpoint_circle(consts["fast_ring_points"]["radius"])
    # contiguous: consecutive points are 8-neighbours, cyclically
    for k in range(16):
        a, b = ring[k], ring[(k + 1) % 16]
        assert max(abs(a[0] - b[0]), abs(a[1] - b[1])) == 1
    # starts at the top and runs clockwise (x right, y down)
    assert ring[0] == (0, -3) and ring[4] == (3, 0) and ring[8] == (0, 3) and ring[12] == (-3, 0)
    for i, j in consts["early_reject_pairs"]["value"]:
        assert ring[i] == (-ring[j][0], -ring[j][1])


def brute_fast(img):
    """Literal Sec. III-D: largest tau >= 0 with 9 contiguous ring pixels all
    > I(p)+tau or all < I(p)-tau, found by trying every tau."""
    dx, dy = oracle.fast_ring()
    h, w = img.shape
    out = np.full((h, w), -1, np.int16)
    im = img.astype(int)
    for y in range(3, h - 3):
        for x in range(3, w - 3):
            c = im[y, x]
            ring = [im[y + dy[k], x + dx[k]] for k in range(16)]
            for tau in range(255, -1, -1):
                b = [v > c + tau for v in ring]
                d = [v < c - tau for v in ring]
                hit = any(all(b[(s + a) % 16] for a in range(9)) or
                          all(d[(s + a) % 16] for a in range(9)) for s in range(16))
                if hit:
                    out[y, x] = tau
                    break
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_fast_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 256, (14, 15)).astype(np.uint8)
    # add structure: a bright blob and a dark blob so corners exist at many taus
    img[4:7, 4:7] = 250
    img[8:10, 9:12] = 3
    assert np.array_equal(oracle.fast_scores(img), brute_fast(img))


def test_fast_isolated_dot_and_flat():
    img = np.full((21, 21), 100, np.uint8)
    assert (oracle.fast_scores(img) == -1).all()
    img[10, 10] = 160
    s = oracle.fast_scores(img)
    assert s[10, 10] == 59           # every ring pixel darker by 60 -> tau = 59
    s[10, 10] = -1
    assert (s == -1).all()           # ring pixels of the dot see one brighter pixel only


def test_fast_straight_edge_has_no_corner():
    img = np.full((20, 20), 50, np.uint8)
    img[:, 10:] = 200
    assert (oracle.fast_scores(img) == -1).all()   # at most 7 contiguous brighter


def test_fast_arc_length_9_vs_8():
    dx, dy = oracle.fast_ring()
    for arc, expect in [(9, 29), (8, -1)]:
        img = np.full((9, 9), 100, np.uint8)
        for k in range(arc):
            img[4 + dy[(k + 5) % 16], 4 + dx[(k + 5) % 16]] = 130 if k else 140
        assert oracle.fast_scores(img)[4, 4] == expect


def test_fast_border_is_not_scored():
    s = oracle.fast_scores(rnd(3, 12, 12))
    inner = s[3:9, 3:9]
    s[3:9, 3:9] = -1
    assert (s == -1).all() and (inner >= -1).all()


# -------------------------------------------------------------- detection ---

def brute_detect(img, cw, ch, k, tmin, border, occ=None, mask=None):
    """Top-k per cell of the strict 3x3 maxima with score >= tmin, by a
    sliding-window maximum and a Python sort."""
    s = oracle.fast_scores(img).astype(int)
    h, w = s.shape
    pad = np.pad(s, 1, constant_values=-1)
    neigh = np.full_like(s, -10)
    for dy, dx in itertools.product((-1, 0, 1), repeat=2):
        if dx or dy:
            neigh = np.maximum(neigh, pad[1 + dy:1 + dy + h, 1 + dx:1 + dx + w])
    cand = (s >= 0) & (s > neigh) & (s >= tmin)
    out = []
    gx, gy = w // cw, h // ch
    for cy in range(gy):
        for cx in range(gx):
            ke = k - (0 if occ is None else int(occ[cy * gx + cx]))
            lst = []
            for y in range(cy * ch, (cy + 1) * ch):
                for x in range(cx * cw, (cx + 1) * cw):
                    if not (border <= x <= w - 1 - border and border <= y <= h - 1 - border):
                        continue
                    if mask is not None and mask[y, x] == 0:
                        continue
                    if cand[y, x]:
                        lst.append((-s[y, x], y, x))
            lst.sort()
            out += [(x, y, -ns) for ns, y, x in lst[:max(ke, 0)]]
    return out


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_detect_loop_equals_one_pass_and_brute_force(k, seed):
    from paper_2609_30459_gb300 import synth
    img = synth.quantize(synth.band_limited_texture(seed, 96, 128, 1.5), None, 0)
    rng = np.random.default_rng(seed)
    occ = rng.integers(0, 3, (96 // 24) * (128 // 20)).astype(np.uint8)
    mask = (rng.random((96, 128)) > 0.1).astype(np.uint8)
    for o, m in [(None, None), (occ, None), (occ, mask)]:
        kp0, s0 = oracle.detect_grid(img, 20, 24, k=k, border=4, occupancy=o, mask=m)
        kp1, s1 = oracle.detect_grid(img, 20, 24, k=k, border=4, occupancy=o, mask=m,
                                     one_pass=True)
        assert np.array_equal(kp0, kp1) and np.array_equal(s0, s1)
        ref = brute_detect(img, 20, 24, k, 5, 4, o, m)
        got = [(int(x), int(y), int(sc)) for (x, y), sc in zip(kp0, s0)]
        assert got == ref


def test_detect_threshold_sequence_stops_early():
    # With a strong corner (score >= 40) in the cell, the k = 1 pick is it,
    # and weaker maxima elsewhere in the cell are not added.
    img = np.full((40, 40), 100, np.uint8)
    img[10, 10] = 200      # score 99
    img[25, 25] = 108      # score 7 (only a corner from threshold 5 on)
    kp, sc = oracle.detect_grid(img, 40, 40, k=2, border=3)
    assert [tuple(p) for p in kp.tolist()] == [(10.0, 10.0), (25.0, 25.0)]
    assert sc.tolist() == [99, 7]
    kp, sc = oracle.detect_grid(img, 40, 40, k=1, border=3)
    assert sc.tolist() == [99]
    kp, sc = oracle.detect_grid(img, 40, 40, k=2, thresholds=(40, 20, 10), border=3)
    assert sc.tolist() == [99]


def test_detect_plateau_is_suppressed_and_ties_ordered():
    img = np.full((30, 60), 100, np.uint8)
    img[10, 10] = img[10, 11] = 180        # equal neighbours suppress each other
    img[20, 40] = img[20, 30] = 180        # equal isolated: order y asc, then x asc
    img[15, 50] = 180
    kp, sc = oracle.detect_grid(img, 60, 30, k=3, border=3)
    assert [tuple(p) for p in kp.tolist()] == [(50.0, 15.0), (30.0, 20.0), (40.0, 20.0)]


def test_detect_occupancy_and_full_cells_only():
    img = np.full((50, 50), 100, np.uint8)
    img[10, 10] = 200
    img[10, 35] = 200
    img[45, 10] = 200       # in the partial bottom row of cells: never detected
    kp, _ = oracle.detect_grid(img, 25, 20, k=1, border=3)
    assert [tuple(p) for p in kp.tolist()] == [(10.0, 10.0), (35.0, 10.0)]
    occ = np.array([1, 0, 0, 0], np.uint8)
    kp, _ = oracle.detect_grid(img, 25, 20, k=1, border=3, occupancy=occ)
    assert [tuple(p) for p in kp.tolist()] == [(35.0, 10.0)]


def test_paper_constants(consts):
    assert list(oracle.THRESHOLDS) == consts["threshold_sequence"]["value"]
    assert oracle.GN_ITERS == consts["gn_iters_per_level"]["value"]
    assert len(oracle.pattern(0)) == consts["pattern_points"]["value"]
