"""A four-camera rig (two stereo pairs with overlapping views of one scene, as
in the paper's four-camera runs, Sec. IV-A): the new keypoints of camera 0 are
matched into every other camera (vio_match_cameras, Sec. III-E's cross-camera
matching with the forward-backward check), from the identity start and from
the model-based start with each camera's extrinsics. Every target against the
FP64 oracle's tracker from the same start; matches near the ground truth."""
import numpy as np
import pytest
import torch

import oracle
from oracle import predict as op
from paper_2609_30459_gb300 import synth
from tests.parity_util import compare_tracks

pytestmark = pytest.mark.gpu

vio = pytest.importorskip("paper_2609_30459_gb300.vio")
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vio.load(build=True)
    oracle.build()


def _rig(seed, w, h):
    """Cameras 0, 1: a stereo pair (disparity 5 + 25 y / h px); cameras 2, 3:
    a second pair whose view is shifted by (24, 8) px and turned by 0.01 rad."""
    scene = synth.PlanarScene(seed, 2048, 2048)
    rng = np.random.default_rng(seed + 1)
    pa = synth.Pose(1.0, 0.0, 0.0, 0.0)
    pb = synth.Pose(1.0, 0.01, 24.0, 8.0)
    imgs = np.stack([scene.render(pa, w, h, None, rng, 2.0),
                     scene.render(pa, w, h, (5.0, 25.0), rng, 2.0),
                     scene.render(pb, w, h, None, rng, 2.0),
                     scene.render(pb, w, h, (5.0, 25.0), rng, 2.0)])
    return scene, pa, pb, imgs


@pytest.mark.parametrize("start", ["identity", "model"])
def test_match_new_keypoints_into_every_camera(start):
    w, h, L = 752, 480, 4
    scene, pa, pb, imgs = _rig(6100, w, h)
    kp, _ = oracle.detect_grid(imgs[0], 37, 32, k=1, border=9)
    n = len(kp)
    p = vio.default_params(n_levels=L)
    ctx = vio.Context(p, w, h, 4)
    pyr = vio.Pyramids(torch.from_numpy(imgs).to(DEV), L)
    ctx.pyramid_build(pyr)
    cap = n + 5                                   # ragged tail
    pts = torch.zeros((cap, 2), device=DEV)
    pts[:n] = torch.from_numpy(kp)
    cnt = torch.tensor([n], dtype=torch.int32, device=DEV)
    # ground truth per target: camera 1 and 3 see x + d(y); camera 2 the
    # similarity map of the second pose
    gt2 = synth.PlanarScene.map_points(pa, pb, kp, w, h, scene.c_tex)
    d = lambda y: 5.0 + 25.0 * y / h
    gts = [kp - np.stack([d(kp[:, 1]), 0 * kp[:, 1]], 1), gt2,
           gt2 - np.stack([d(gt2[:, 1]), 0 * gt2[:, 1]], 1)]
    init = None
    starts = [None, None, None]
    if start == "model":
        # each target's start from the rig's calibration (pinhole f = 500 px,
        # stereo baseline 1) and the plane's inverse depth (the backend's
        # depth; here the generator's): camera 1 is camera 0 shifted by the
        # baseline, so x moves by the disparity f b rho(y) of the plane, whose
        # inverse depth is affine in y; camera 2 is the second pose; camera 3
        # the second pose, then its baseline
        f, base = 500.0, 1.0
        K, R, t, rho = op.similarity_rig(pa, pb, f, w, h)
        pat = oracle.pattern()
        s1, _ = op.predict_warp(K, K, np.eye(3), np.array([-base, 0.0, 0.0]), kp,
                                d(kp[:, 1]) / (f * base), pat)
        s2, _ = op.predict_warp(K, K, R, t, kp, np.full(n, rho), pat)
        s3 = s2.copy()
        s3[:, 0] -= d(s2[:, 1])
        for j, sj in enumerate((s1, s2, s3)):
            row = np.zeros((cap, 3), np.float32)
            row[:, :2] = pts.cpu().numpy()
            row[:n] = sj
            starts[j] = row
        init = torch.from_numpy(np.stack(starts)).to(DEV).contiguous()
    match = torch.zeros((3, cap, 2), device=DEV)
    status = torch.zeros((3, cap), dtype=torch.uint8, device=DEV)
    fbd = torch.zeros((3, cap), device=DEV)
    ctx.match_cameras(pyr, pyr.batch(0, 1, 1), pyr.batch(1, 1, 3), pts, cnt, cap, match, status,
                      fb_dist=fbd, init=init)
    torch.cuda.synchronize()
    opyr = [oracle.pyramid(im, L) for im in imgs]
    for j in range(3):
        ini = None if starts[j] is None else starts[j][:n]
        ref = oracle.track(opyr[0], opyr[j + 1], kp, init=ini, fb_max_dist=p.fb_max_dist,
                           n_threads=8)
        s = compare_tracks(match[j, :n].cpu().numpy(), status[j, :n].cpu().numpy(), ref,
                           p.fb_max_dist)
        print(start, j, s)
        assert (status[j, n:] == 255).all()
        ok = status[j, :n].cpu().numpy() == 0
        err = np.abs(match[j, :n].cpu().numpy()[ok] - gts[j][ok]).max(1)
        assert s["agree"] >= 0.999, (j, s)           # the oracle's tracker, same start
        # the identity start reaches the stereo partner; the second pair, 25 px
        # and 0.01 rad away, needs the model-based start (from the identity
        # few of its tracks pass the check, some at a wrong optimum)
        if start == "model" or j == 0:
            assert ok.mean() > 0.6, (j, s)
            assert (err < 0.5).mean() > 0.95, (j, np.percentile(err, 99))
    ctx.close()
