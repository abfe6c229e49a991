"""Oracle of the model-based start of a track (Sec. III-E). TEST
INFRASTRUCTURE ONLY.

The paper starts each track's warp by projecting the sample pattern into the
target image through the camera model, with the predicted pose and the
keypoint's inverse depth. Restated here in FP64 for a pinhole camera:

* back-projection of a source pixel u with inverse depth rho:
  P = (1 / rho) K_src^-1 [u, 1];
* the predicted relative pose (R, t) maps it to the target camera:
  P' = R P + t;
* projection: u' = (fx' P'x / P'z + cx', fy' P'y / P'z + cy').

The start warp (t0, theta0) of keypoint p: t0 = the projection of p itself;
every pattern point p + x_i is projected with the keypoint's inverse depth (a
fronto-parallel patch) to y_i, and theta0 is the angle of the least-squares
rotation taking the offsets x_i onto y_i - t0 (the angle of
sum_i x_i^T y~_i + i * sum_i x_i x y~_i, with y~_i = y_i - t0). A keypoint
whose back-projected point, or any projected pattern point, does not lie in
front of the target camera (P'z <= 0), or with rho <= 0, has no prediction:
its start is the identity (t0 = p, theta0 = 0) and valid = False.
"""
from __future__ import annotations

import numpy as np


def project(K_src, K_dst, R, t, u, rho):
    """Projection of source pixel(s) u (..., 2) at inverse depth rho (...)
    into the target camera: (u' (..., 2), depth P'z (...))."""
    fx, fy, cx, cy = (float(v) for v in K_src)
    gx, gy, dx, dy = (float(v) for v in K_dst)
    u = np.asarray(u, np.float64)
    rho = np.asarray(rho, np.float64)
    z = 1.0 / rho
    P = np.stack([(u[..., 0] - cx) / fx * z, (u[..., 1] - cy) / fy * z, z], -1)
    Q = P @ np.asarray(R, np.float64).reshape(3, 3).T + np.asarray(t, np.float64).reshape(3)
    out = np.stack([gx * Q[..., 0] / Q[..., 2] + dx, gy * Q[..., 1] / Q[..., 2] + dy], -1)
    return out, Q[..., 2]


def predict_warp(K_src, K_dst, R, t, pts, inv_depth, pattern):
    """Start warps (n, 3) = (tx, ty, theta) and validity (n,) of keypoints pts
    (n, 2) with inverse depths (n,), for pattern offsets (m, 2)."""
    pts = np.asarray(pts, np.float64).reshape(-1, 2)
    rho = np.asarray(inv_depth, np.float64).reshape(-1)
    x = np.asarray(pattern, np.float64).reshape(-1, 2)
    n = len(pts)
    out = np.zeros((n, 3))
    out[:, :2] = pts
    valid = np.zeros(n, bool)
    for i in range(n):
        if not rho[i] > 0:
            continue
        c, zc = project(K_src, K_dst, R, t, pts[i], rho[i])
        y, zy = project(K_src, K_dst, R, t, pts[i] + x, np.full(len(x), rho[i]))
        if not (zc > 0 and np.all(zy > 0)):
            continue
        d = y - c
        dot = float(np.sum(x[:, 0] * d[:, 0] + x[:, 1] * d[:, 1]))
        cross = float(np.sum(x[:, 0] * d[:, 1] - x[:, 1] * d[:, 0]))
        out[i] = (c[0], c[1], np.arctan2(cross, dot))
        valid[i] = True
    return out, valid


def similarity_rig(pose_a, pose_b, f, w, h):
    """Pinhole form of the synthetic planar scene's similarity poses
    (synth.Pose: texture = c_tex + s R(th) (u - c) + t, c the image centre):
    camera a looks at the textured plane fronto-parallel from depth f * s_a,
    rotated by th_a about its axis. Returns (K, R, t, rho): the intrinsics
    shared by both frames, the relative pose b <- a and the inverse depth of
    every point of the plane in camera a."""
    c = ((w - 1) / 2.0, (h - 1) / 2.0)
    K = (f, f, c[0], c[1])

    def rz(a):
        ca, sa = np.cos(a), np.sin(a)
        return np.array([[ca, -sa, 0.0], [sa, ca, 0.0], [0.0, 0.0, 1.0]])

    Ra, Rb = rz(pose_a.th), rz(pose_b.th)
    Ca = np.array([pose_a.tx, pose_a.ty, -f * pose_a.s])
    Cb = np.array([pose_b.tx, pose_b.ty, -f * pose_b.s])
    R = Rb.T @ Ra
    t = Rb.T @ (Ca - Cb)
    return K, R, t, 1.0 / (f * pose_a.s)
