"""GPU parity of the model-based start of a track (vio_predict_warp, Sec.
III-E) against the FP64 oracle (oracle.predict), and of tracks started there
against the oracle's tracker started at the oracle's prediction."""
import numpy as np
import pytest
import torch

import oracle
from oracle import predict as op
from paper_2609_30459_gb300 import synth
from tests.parity_util import FLOW_TOL, THETA_TOL, compare_tracks

pytestmark = pytest.mark.gpu

vio = pytest.importorskip("paper_2609_30459_gb300.vio")
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vio.load(build=True)
    oracle.build()


def _rot(rng, scale):
    a = rng.normal(0, scale, 3)
    th = np.linalg.norm(a)
    k = a / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * Kx @ Kx


def test_predict_matches_oracle():
    rng = np.random.default_rng(11)
    n_img, cap, w, h = 3, 200, 1280, 720
    ks, kd = (700.0, 690.0, 640.5, 360.25), (650.0, 655.0, 630.0, 355.0)
    poses = np.zeros((n_img, 12), np.float32)
    for i in range(n_img):
        poses[i, :9] = _rot(rng, 0.05).reshape(-1)
        poses[i, 9:] = rng.normal(0, 0.3, 3)
    pts = rng.uniform([0, 0], [w, h], (n_img, cap, 2)).astype(np.float32)
    rho = rng.uniform(0.05, 0.5, (n_img, cap)).astype(np.float32)
    rho[:, ::17] = -0.1                               # no depth: identity start
    counts = np.array([cap, 131, 0], np.int32)
    init = torch.full((n_img, cap, 3), -5.0, device=DEV)
    valid = torch.full((n_img, cap), 7, dtype=torch.uint8, device=DEV)
    vio.predict_warp(ks, kd, torch.from_numpy(poses).to(DEV), torch.from_numpy(pts).to(DEV),
                     torch.from_numpy(rho).to(DEV), torch.from_numpy(counts).to(DEV), cap,
                     n_img, init, valid)
    torch.cuda.synchronize()
    g, gv = init.cpu().numpy(), valid.cpu().numpy()
    pat = oracle.pattern()
    for i in range(n_img):
        c = counts[i]
        ref, rv = op.predict_warp(ks, kd, poses[i, :9].astype(np.float64).reshape(3, 3),
                                  poses[i, 9:].astype(np.float64), pts[i, :c], rho[i, :c], pat)
        assert np.array_equal(gv[i, :c].astype(bool), rv)
        assert (gv[i, c:] == 0).all()
        assert (g[i, c:] == -5.0).all()                 # slots past the count untouched
        assert np.abs(g[i, :c, :2] - ref[:, :2]).max(initial=0) < FLOW_TOL
        assert np.abs(g[i, :c, 2] - ref[:, 2]).max(initial=0) < THETA_TOL
        assert rv.sum() > 0.8 * c if c else True


def test_tracks_from_the_prediction_match_oracle():
    """Two frames of a 40 px-motion sequence: the GPU tracker started at the
    GPU prediction against the oracle's tracker started at the oracle's; and
    the prediction keeps more tracks near the ground truth than the identity
    start."""
    w, h, L = 640, 480, 5
    seq = synth.make_sequence(8101, 2, w, h, 1, max_motion=40.0, tex_size=2048)
    a, b = seq.poses[0][0], seq.poses[1][0]
    K, R, t, rho = op.similarity_rig(a, b, 500.0, w, h)
    imgs = seq.frames[:, 0]
    kp, _ = oracle.detect_grid(imgs[0], 32, 32, k=1, border=9)
    n = len(kp)
    p = vio.default_params(n_levels=L)
    ctx = vio.Context(p, w, h, 2)
    pyr = vio.Pyramids(torch.from_numpy(np.ascontiguousarray(imgs)).to(DEV), L)
    ctx.pyramid_build(pyr)
    pose = torch.from_numpy(np.concatenate([R.reshape(-1), t]).astype(np.float32)[None]).to(DEV)
    pts = torch.from_numpy(kp).to(DEV)[None].contiguous()
    d_rho = torch.full((1, n), rho, dtype=torch.float32, device=DEV)
    init = torch.empty((1, n, 3), device=DEV)
    vio.predict_warp(K, K, pose, pts, d_rho, None, n, 1, init)
    out = torch.empty((1, n, 3), device=DEV)
    st = torch.empty((1, n), dtype=torch.uint8, device=DEV)
    cnt = torch.tensor([n], dtype=torch.int32, device=DEV)
    ctx.track_patches(pyr, pyr.batch(0, 1, 1), pyr.batch(1, 1, 1), pts, cnt, n, out, st,
                      init=init)
    out0 = torch.empty_like(out)
    st0 = torch.empty_like(st)
    ctx.track_patches(pyr, pyr.batch(0, 1, 1), pyr.batch(1, 1, 1), pts, cnt, n, out0, st0)
    torch.cuda.synchronize()
    ref_init, _ = op.predict_warp(K, K, R, t, kp, np.full(n, rho), oracle.pattern())
    opyr = [oracle.pyramid(im, L) for im in imgs]
    ref = oracle.track(opyr[0], opyr[1], kp, init=ref_init.astype(np.float32), n_threads=8)
    compare_tracks(out[0, :, :2].cpu().numpy(), st[0].cpu().numpy(), ref, p.fb_max_dist,
                   g_theta=out[0, :, 2].cpu().numpy())
    gt = synth.PlanarScene.map_points(a, b, kp, w, h, seq.c_tex)
    good = lambda o, s: ((s == 0) & (np.abs(o[:, :2] - gt).max(1) < 0.5)).mean()
    g_pred = good(out[0].cpu().numpy(), st[0].cpu().numpy())
    g_id = good(out0[0].cpu().numpy(), st0[0].cpu().numpy())
    print(f"within 0.5 px of the truth: model-based start {g_pred:.3f}, identity {g_id:.3f}")
    assert g_pred > g_id + 0.2 and g_pred > 0.3
    ctx.close()


def test_predict_rejects_bad_intrinsics():
    z = torch.zeros(16, device=DEV)
    with pytest.raises(vio.VioError):
        vio.predict_warp((0.0, 1.0, 0.0, 0.0), (1.0, 1.0, 0.0, 0.0), z, z, z, None, 1, 1, z)
