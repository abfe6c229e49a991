"""Seeded synthetic inputs shaped like the paper's workloads.

The paper evaluates on recorded datasets (EuRoC, TUM-VI, MSD, Hilti; Sec.
IV-A) that are not available here. These generators stand in for them with
seeded, synthetic stereo sequences of the same kind: a band-limited noise
texture (uniform noise filtered by a Gaussian of sigma 2 px, rescaled to mean
128 and standard deviation 40) seen by a camera that moves smoothly over a
plane, rendered with cubic-spline sampling, plus N(0, 2^2) sensor noise per
image, rounded half up and clipped to uint8. The right image of a stereo pair
sees the scene shifted by a disparity that is linear in the row.

This module holds no arithmetic of the frontend itself (no pyramid, detector
or tracker): both the CUDA library's tests and the CPU oracle's tests take
their inputs from here.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy import ndimage

__all__ = ["Pose", "PlanarScene", "Sequence", "make_sequence", "stereo_pair_small_motion",
           "band_limited_texture", "quantize"]


def band_limited_texture(seed: int, h: int, w: int, sigma: float = 2.0, mean: float = 128.0,
                         std: float = 40.0) -> np.ndarray:
    """U[0,255] noise, Gaussian-filtered (periodic), rescaled to mean/std (FP64)."""
    rng = np.random.default_rng(seed)
    t = ndimage.gaussian_filter(rng.uniform(0.0, 255.0, (h, w)), sigma, mode="wrap")
    sd = t.std()
    t = (t - t.mean()) / sd if sd > 0 else np.zeros_like(t)
    return mean + std * t


def quantize(v: np.ndarray, rng: np.random.Generator | None, noise_sigma: float) -> np.ndarray:
    """Additive Gaussian noise (DN), round half up, clip to [0, 255] -> uint8."""
    if rng is not None and noise_sigma > 0:
        v = v + rng.normal(0.0, noise_sigma, v.shape)
    return np.clip(np.floor(v + 0.5), 0, 255).astype(np.uint8)


@dataclass
class Pose:
    """Camera pose over the textured plane: image pixel x maps to texture
    coordinate c_tex + s * R(th) (x - c_img) + (tx, ty)."""
    s: float = 1.0
    th: float = 0.0
    tx: float = 0.0
    ty: float = 0.0

    def matrix(self, c_img, c_tex) -> np.ndarray:
        c, s_ = np.cos(self.th), np.sin(self.th)
        A = self.s * np.array([[c, -s_], [s_, c]])
        b = np.array(c_tex, float) + np.array([self.tx, self.ty]) - A @ np.array(c_img, float)
        M = np.eye(3)
        M[:2, :2] = A
        M[:2, 2] = b
        return M


class PlanarScene:
    """A periodic band-limited texture of size (tex_h, tex_w) and a renderer."""

    def __init__(self, seed: int, tex_h: int = 1024, tex_w: int = 1024, sigma: float = 2.0):
        self.seed = seed
        self.tex = band_limited_texture(seed, tex_h, tex_w, sigma)
        self._coef = ndimage.spline_filter(self.tex, order=3, mode="grid-wrap")
        self.c_tex = (tex_w / 2.0, tex_h / 2.0)

    def sample(self, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        """Texture values at float texture coordinates (cubic spline, periodic)."""
        return ndimage.map_coordinates(self._coef, [Y, X], order=3, mode="grid-wrap",
                                       prefilter=False)

    def render(self, pose: Pose, w: int, h: int, disparity: tuple[float, float] | None = None,
               rng: np.random.Generator | None = None, noise_sigma: float = 2.0,
               exact: bool = False) -> np.ndarray:
        """Render a w x h image. disparity=(d0, d1): this camera sees the left
        camera's pixel (x + d0 + d1 * y / h, y). exact=True returns the FP64
        image without noise or quantisation."""
        ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
        if disparity is not None:
            xs = xs + disparity[0] + disparity[1] * ys / h
        M = pose.matrix(((w - 1) / 2.0, (h - 1) / 2.0), self.c_tex)
        X = M[0, 0] * xs + M[0, 1] * ys + M[0, 2]
        Y = M[1, 0] * xs + M[1, 1] * ys + M[1, 2]
        v = self.sample(X, Y)
        return v if exact else quantize(v, rng, noise_sigma)

    @staticmethod
    def map_points(pose_a: Pose, pose_b: Pose, pts: np.ndarray, w: int, h: int,
                   c_tex) -> np.ndarray:
        """Ground truth: pixel positions in camera pose_a -> the pixels of pose_b
        that see the same scene point."""
        c_img = ((w - 1) / 2.0, (h - 1) / 2.0)
        Ma = pose_a.matrix(c_img, c_tex)
        Mb = pose_b.matrix(c_img, c_tex)
        P = np.concatenate([np.asarray(pts, float).reshape(-1, 2),
                            np.ones((len(pts), 1))], axis=1)
        Q = (np.linalg.inv(Mb) @ Ma @ P.T).T
        return Q[:, :2]


@dataclass
class Sequence:
    frames: np.ndarray                 # (F, C, H, W) uint8; cameras 2p, 2p+1 are a stereo pair
    poses: list[list[Pose]]            # per frame, per stereo pair
    disparity: tuple[float, float]
    scene_seed: int
    c_tex: tuple[float, float] = field(default=(0.0, 0.0))

    @property
    def shape(self):
        return self.frames.shape


def _trajectory(rng: np.random.Generator, n_frames: int):
    """Sum of 3 sinusoids per degree of freedom (tx, ty, theta, log scale)."""
    t = np.arange(n_frames, dtype=np.float64)
    out = []
    for amp in (1.0, 1.0, 0.004, 0.0015):
        f = rng.uniform(0.004, 0.03, 3)            # cycles per frame
        ph = rng.uniform(0, 2 * np.pi, 3)
        a = amp * rng.uniform(0.5, 1.0, 3) / (2 * np.pi * f)
        out.append((a[None, :] * np.sin(2 * np.pi * f[None, :] * t[:, None] + ph)).sum(1))
    return np.stack(out, 1)  # (F, 4)


def make_sequence(seed: int, n_frames: int, w: int, h: int, n_pairs: int = 1,
                  max_motion: float = 15.0, disparity=(5.0, 25.0), noise_sigma: float = 2.0,
                  tex_size: int = 4096) -> Sequence:
    """A stereo sequence over a planar texture: per-frame image motion of at
    most ``max_motion`` px (at the image corners), a smooth random trajectory
    per stereo pair, right images at disparity d0 + d1 * y / h."""
    scene = PlanarScene(seed, tex_size, tex_size)
    rng = np.random.default_rng(seed + 7919)
    corners = np.array([[0, 0], [w - 1, 0], [0, h - 1], [w - 1, h - 1]], float)
    frames = np.zeros((n_frames, 2 * n_pairs, h, w), np.uint8)
    poses: list[list[Pose]] = [[] for _ in range(n_frames)]
    for pair in range(n_pairs):
        traj = _trajectory(rng, n_frames)
        base = np.array([pair * tex_size / 2.0, pair * tex_size / 3.0, 0.0, 0.0])

        def pose_at(f, k):
            d = base + k * traj[f]
            return Pose(s=float(np.exp(d[3])), th=float(d[2]), tx=float(d[0]), ty=float(d[1]))

        # scale the trajectory so that the largest per-frame corner motion is max_motion
        peak = 0.0
        for f in range(1, n_frames):
            q = PlanarScene.map_points(pose_at(f - 1, 1.0), pose_at(f, 1.0), corners, w, h,
                                       scene.c_tex)
            peak = max(peak, float(np.abs(q - corners).max()))
        k = max_motion / peak if peak > 0 else 1.0
        for f in range(n_frames):
            p = pose_at(f, k)
            poses[f].append(p)
            frames[f, 2 * pair] = scene.render(p, w, h, None, rng, noise_sigma)
            frames[f, 2 * pair + 1] = scene.render(p, w, h, disparity, rng, noise_sigma)
    return Sequence(frames, poses, tuple(disparity), seed, scene.c_tex)


def stereo_pair_small_motion(seed: int, w: int = 752, h: int = 480, max_t: float = 3.0,
                             max_deg: float = 1.0, disparity=(5.0, 25.0),
                             noise_sigma: float = 2.0):
    """One stereo pair at t and the next pair at t+1 under a random SE(2)
    motion with |t| <= max_t px and |theta| <= max_deg degrees. Returns a dict
    with images (2, 2, h, w) [time, camera], the motion and the scene."""
    tex = 1 << int(np.ceil(np.log2(max(w, h) + 256)))
    scene = PlanarScene(seed, tex, tex)
    rng = np.random.default_rng(seed + 104729)
    ang = np.deg2rad(rng.uniform(-max_deg, max_deg))
    r = rng.uniform(0, max_t)
    phi = rng.uniform(0, 2 * np.pi)
    p0 = Pose()
    p1 = Pose(1.0, float(ang), float(r * np.cos(phi)), float(r * np.sin(phi)))
    imgs = np.zeros((2, 2, h, w), np.uint8)
    for ti, p in enumerate((p0, p1)):
        imgs[ti, 0] = scene.render(p, w, h, None, rng, noise_sigma)
        imgs[ti, 1] = scene.render(p, w, h, disparity, rng, noise_sigma)
    return {"images": imgs, "poses": (p0, p1), "scene": scene, "disparity": disparity}
