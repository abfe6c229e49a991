"""Pins of the model-based start oracle (oracle.predict, Sec. III-E: the warp
starts at the projection of the pattern through the camera model with the
predicted pose and inverse depth).

Checked against things other than its own formula: the generator's
ground-truth point map of the synthetic planar scene (a similarity written as
3x3 matrices, synth.PlanarScene.map_points), closed forms for the identity,
a roll about the optical axis and a pure depth change, and the tracker: a
start at the prediction sits at the optimum on a noise-free render, where the
identity start at 40 px of motion does not converge."""
import numpy as np
import pytest

import oracle
from oracle import predict as op
from paper_2609_30459_gb300 import synth

PAT = None


def _pattern():
    global PAT
    if PAT is None:
        oracle.build()
        PAT = oracle.pattern()
    return PAT


def test_identity_pose_keeps_the_keypoint():
    K = (500.0, 480.0, 320.0, 240.0)
    pts = np.array([[10.5, 20.25], [320.0, 240.0], [600.0, 470.0]])
    w, v = op.predict_warp(K, K, np.eye(3), np.zeros(3), pts, np.full(3, 1e-3), _pattern())
    assert v.all()
    assert np.abs(w[:, :2] - pts).max() < 1e-9
    assert np.abs(w[:, 2]).max() < 1e-12


def test_roll_about_the_optical_axis():
    # R = rotation by phi about z: u' - c = R(phi) (u - c), theta = phi (fx = fy)
    f, c = 600.0, np.array([400.0, 300.0])
    K = (f, f, c[0], c[1])
    phi = 0.07
    R = np.array([[np.cos(phi), -np.sin(phi), 0], [np.sin(phi), np.cos(phi), 0], [0, 0, 1]])
    pts = np.array([[100.0, 50.0], [400.0, 300.0], [700.0, 580.0]])
    w, v = op.predict_warp(K, K, R, np.zeros(3), pts, np.full(3, 0.01), _pattern())
    Rp = np.array([[np.cos(phi), -np.sin(phi)], [np.sin(phi), np.cos(phi)]])
    exp = c + (pts - c) @ Rp.T
    assert v.all()
    assert np.abs(w[:, :2] - exp).max() < 1e-9
    assert np.abs(w[:, 2] - phi).max() < 1e-12


def test_depth_change_scales_about_the_principal_point():
    # moving the camera towards a fronto-parallel point at depth z by dz scales
    # image offsets by z / (z - dz); a pure zoom has no rotation
    f, c = 500.0, np.array([320.0, 240.0])
    K = (f, f, c[0], c[1])
    z, dz = 100.0, 20.0
    pts = np.array([[20.0, 30.0], [500.0, 400.0]])
    w, v = op.predict_warp(K, K, np.eye(3), np.array([0.0, 0.0, -dz]), pts,
                           np.full(2, 1.0 / z), _pattern())
    assert v.all()
    assert np.abs(w[:, :2] - (c + (pts - c) * z / (z - dz))).max() < 1e-9
    assert np.abs(w[:, 2]).max() < 1e-12


def test_matches_the_generators_ground_truth_map():
    rng = np.random.default_rng(3)
    w_, h_ = 752, 480
    for _ in range(20):
        a = synth.Pose(rng.uniform(0.8, 1.2), rng.uniform(-0.3, 0.3), *rng.uniform(-50, 50, 2))
        b = synth.Pose(a.s * rng.uniform(0.9, 1.1), a.th + rng.uniform(-0.05, 0.05),
                       a.tx + rng.uniform(-30, 30), a.ty + rng.uniform(-30, 30))
        K, R, t, rho = op.similarity_rig(a, b, rng.uniform(300, 900), w_, h_)
        pts = rng.uniform([0, 0], [w_ - 1, h_ - 1], (25, 2))
        gt = synth.PlanarScene.map_points(a, b, pts, w_, h_, (2048.0, 2048.0))
        pw, v = op.predict_warp(K, K, R, t, pts, np.full(len(pts), rho), _pattern())
        assert v.all()
        assert np.abs(pw[:, :2] - gt).max() < 1e-8
        # a similarity turns every offset by th_a - th_b
        assert np.abs(pw[:, 2] - (a.th - b.th)).max() < 1e-9


def test_points_behind_the_target_camera_have_no_prediction():
    K = (500.0, 500.0, 320.0, 240.0)
    pts = np.array([[100.0, 100.0], [200.0, 200.0]])
    # target camera 20 units in front of the point along its axis: P'z < 0
    w, v = op.predict_warp(K, K, np.eye(3), np.array([0.0, 0.0, -20.0]), pts,
                           np.array([0.1, -1.0]), _pattern())
    assert not v.any()
    assert np.array_equal(w[:, :2], pts) and (w[:, 2] == 0).all()


def test_start_at_the_prediction_is_the_tracking_optimum():
    """Two frames of the generator 36 px apart under an SE(2) motion (the
    warp model of the tracker: translation and a rotation of 0.02 rad),
    rendered without noise: from the model-based start the track ends within
    0.02 px of it and of the ground truth; from the identity start most
    tracks do not reach it (keypoints 100 px inside the frame, so that the
    coarsest level's pattern, 7 px there, stays inside the target)."""
    w_, h_, L = 640, 480, 4
    scene = synth.PlanarScene(17, 2048, 2048)
    a = synth.Pose(1.0, 0.0, 0.0, 0.0)
    b = synth.Pose(1.0, 0.02, 30.0, -20.0)
    imgs = [scene.render(p_, w_, h_, None, None, 0.0) for p_ in (a, b)]
    pyr = [oracle.pyramid(im, L) for im in imgs]
    kp, _ = oracle.detect_grid(imgs[0], 48, 48, k=1, border=100)
    K, R, t, rho = op.similarity_rig(a, b, 500.0, w_, h_)
    init, v = op.predict_warp(K, K, R, t, kp, np.full(len(kp), rho), _pattern())
    assert v.all() and len(kp) > 30
    gt = synth.PlanarScene.map_points(a, b, kp, w_, h_, scene.c_tex)
    r = oracle.track(pyr[0], pyr[1], kp, init=init.astype(np.float32), fb=True, n_threads=4)
    ok = r["status"] == 0
    assert ok.mean() > 0.9
    assert np.abs(r["warp"][ok, :2] - init[ok, :2]).max() < 0.02
    assert np.abs(r["warp"][ok, :2] - gt[ok]).max() < 0.02
    r0 = oracle.track(pyr[0], pyr[1], kp, fb=True, n_threads=4)
    good0 = (r0["status"] == 0) & (np.abs(r0["warp"][:, :2] - gt).max(1) < 0.05)
    assert good0.mean() < 0.5
