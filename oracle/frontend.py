"""Oracle of the per-frame frontend (Sec. III-B). TEST INFRASTRUCTURE ONLY.

Stage order per frame, as the paper records it: pyramid, temporal tracking,
detection, cross-camera matching. State per stereo stream: a keypoint list per
camera (float32 positions and int ids) and the next id.

* Temporal tracking: every camera's keypoints from its previous pyramid to
  its current one, identity start, with the forward-backward check; tracks
  with status OK survive, in order, at their tracked position.
* Detection on camera 0 (level 0), with each cell's count of surviving
  camera-0 tracks counted against k (the mask and cell buffers of Sec. III-B).
* Matching: the new keypoints from camera 0 to camera 1 of the same frame,
  identity start, with the forward-backward check.
* New lists: camera 0 = survivors ++ new; camera 1 = survivors ++ the new
  keypoints whose match is OK, at the matched position; both truncated to the
  capacity. New ids are next_id + rank; next_id grows by the number detected.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import detect_grid, pyramid, track


@dataclass
class Params:
    n_levels: int = 4
    round_mode: int = 0
    gn_iters: int = 5
    pattern_id: int = 0
    cell_w: int = 50
    cell_h: int = 50
    k: int = 1
    thresholds: tuple = (40, 20, 10, 5)
    border: int = 9
    fb_max_dist: float = 0.2


@dataclass
class StreamState:
    xy: list = field(default_factory=lambda: [np.zeros((0, 2), np.float32)] * 2)
    ids: list = field(default_factory=lambda: [np.zeros(0, np.int32)] * 2)
    next_id: int = 0
    pyr: list | None = None          # previous frame's pyramids per camera


def occupancy(xy: np.ndarray, w: int, h: int, cw: int, ch: int) -> np.ndarray:
    """Per-cell counts of positions, saturating at 255 (cell raster order)."""
    gx, gy = w // cw, h // ch
    occ = np.zeros(gx * gy, np.int64)
    for x, y in np.asarray(xy, np.float64):
        if x < 0 or y < 0:
            continue
        cx, cy = int(np.floor(x / cw)), int(np.floor(y / ch))
        if cx < gx and cy < gy:
            occ[cy * gx + cx] += 1
    return np.minimum(occ, 255).astype(np.uint8)


def step(state: StreamState, frame: np.ndarray, p: Params, capacity: int,
         n_threads: int = 1) -> dict:
    """One frame (frame: (2, h, w) uint8) for one stream; updates `state`."""
    h, w = frame.shape[1:]
    pyrs = [pyramid(frame[c], p.n_levels, p.round_mode) for c in range(2)]
    surv_xy, surv_id, trk = [], [], []
    for c in range(2):
        xy, ids = state.xy[c], state.ids[c]
        if state.pyr is not None and len(xy):
            r = track(state.pyr[c], pyrs[c], xy, gn_iters=p.gn_iters, pattern_id=p.pattern_id,
                      fb=True, fb_max_dist=p.fb_max_dist, n_threads=n_threads)
            ok = r["status"] == 0
            surv_xy.append(r["warp"][ok, :2].astype(np.float32))
            surv_id.append(ids[ok])
            trk.append(r)
        else:
            surv_xy.append(np.zeros((0, 2), np.float32))
            surv_id.append(np.zeros(0, np.int32))
            trk.append(None)
    occ = occupancy(surv_xy[0], w, h, p.cell_w, p.cell_h)
    new_xy, new_sc = detect_grid(frame[0], p.cell_w, p.cell_h, k=p.k, thresholds=p.thresholds,
                                 border=p.border, occupancy=occ)
    new_id = (state.next_id + np.arange(len(new_xy))).astype(np.int32)
    if len(new_xy):
        m = track(pyrs[0], pyrs[1], new_xy, gn_iters=p.gn_iters, pattern_id=p.pattern_id,
                  fb=True, fb_max_dist=p.fb_max_dist, n_threads=n_threads)
    else:
        m = {"status": np.zeros(0, np.uint8), "warp": np.zeros((0, 3)),
             "fb_dist": np.zeros(0), "margin": np.zeros(0)}
    mok = m["status"] == 0
    state.xy = [np.concatenate([surv_xy[0], new_xy])[:capacity],
                np.concatenate([surv_xy[1], m["warp"][mok, :2].astype(np.float32)])[:capacity]]
    state.ids = [np.concatenate([surv_id[0], new_id])[:capacity],
                 np.concatenate([surv_id[1], new_id[mok]])[:capacity]]
    state.next_id += len(new_xy)
    state.pyr = pyrs
    return {"track": trk, "occupancy": occ, "new_xy": new_xy, "new_score": new_sc,
            "match": m}
