"""Oracle of the per-frame frontend (Sec. III-B). TEST INFRASTRUCTURE ONLY.

Stage order per frame, as the paper records it: pyramid, temporal tracking,
detection, cross-camera matching. State per stereo stream: a keypoint list per
camera (float32 positions and int ids) and the next id.

* Temporal tracking: every camera's keypoints from its previous pyramid to
  its current one, identity start, with the forward-backward check; tracks
  with status OK survive, in order, at their tracked position.
* With the learned initializer (not in the paper; ``NetCfg``): first the
  network's proposal (flow, confidence) for every keypoint; where the
  confidence reaches the gate, the track over levels start_level..0 from
  p + flow; every keypoint without a proposal above the gate, or whose
  proposed track does not end OK, or has not converged (its last level-0
  Gauss-Newton step moved the pattern by more than max_last_step px, when
  that is > 0), is tracked as above.
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

from . import detect_grid, initnet, pyramid, track


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
class NetCfg:
    params: dict                     # network parameters (weights as BF16 values)
    level_a: int = 2
    level_b: int = 3
    start_level: int = 1
    min_conf: float = 0.5
    max_last_step: float = 1e-3      # convergence gate (px), <= 0: none


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


def proposals(net: NetCfg, prev, cur, xy):
    """(flow (n,2) level-0 px, confidence (n,)) of the network, in its own
    precision (BF16 activations)."""
    flow = np.zeros((len(xy), 2))
    conf = np.zeros(len(xy))
    for i, (x, y) in enumerate(np.asarray(xy, np.float32)):
        o = initnet.forward(net.params, initnet.extract(prev, cur, float(x), float(y),
                                                        net.level_a, net.level_b),
                            act_bf16=True)
        flow[i] = o[0] * initnet.SCALE, o[1] * initnet.SCALE
        conf[i] = initnet.sigmoid(o[2])
    return flow, conf


def temporal(prev, cur, xy, p: Params, net: NetCfg | None = None, n_threads: int = 1) -> dict:
    """Temporal tracking of one camera's keypoints (previous -> current
    pyramid). Returns status, warp, fb_dist, margin per keypoint and, with a
    network, the proposals, which keypoints were tracked from them
    (``learned``), and the two track results with their keypoint indices."""
    kw = dict(gn_iters=p.gn_iters, pattern_id=p.pattern_id, fb=True,
              fb_max_dist=p.fb_max_dist, n_threads=n_threads)
    if net is None:
        return track(prev, cur, xy, **kw)
    xy = np.asarray(xy, np.float32)
    n = len(xy)
    flow, conf = proposals(net, prev, cur, xy)
    out = {"status": np.zeros(n, np.uint8), "warp": np.zeros((n, 3)), "fb_dist": np.zeros(n),
           "margin": np.zeros(n), "last_step": np.zeros(n), "flow": flow, "conf": conf,
           "learned": np.zeros(n, bool)}
    gate = np.where(conf >= net.min_conf)[0]
    top = net.start_level + 1
    res_l = None
    if len(gate):
        init = np.zeros((len(gate), 3), np.float32)
        init[:, :2] = (xy[gate] + flow[gate]).astype(np.float32)
        res_l = track(prev[:top], cur[:top], xy[gate], init=init, **kw)
        keep = res_l["status"] == 0
        if net.max_last_step > 0:
            keep &= res_l["last_step"] <= net.max_last_step
        ok = gate[keep]
        out["learned"][ok] = True
        for k in ("status", "warp", "fb_dist", "margin", "last_step"):
            out[k][ok] = res_l[k][keep]
    rest = np.where(~out["learned"])[0]
    res_p = track(prev, cur, xy[rest], **kw) if len(rest) else None
    if res_p is not None:
        for k in ("status", "warp", "fb_dist", "margin", "last_step"):
            out[k][rest] = res_p[k]
    out["learned_track"] = (gate, res_l)
    out["plain_track"] = (rest, res_p)
    return out


def step(state: StreamState, frame: np.ndarray, p: Params, capacity: int,
         n_threads: int = 1, net: NetCfg | None = None) -> dict:
    """One frame (frame: (2, h, w) uint8) for one stream; updates `state`."""
    h, w = frame.shape[1:]
    pyrs = [pyramid(frame[c], p.n_levels, p.round_mode) for c in range(2)]
    surv_xy, surv_id, trk = [], [], []
    for c in range(2):
        xy, ids = state.xy[c], state.ids[c]
        if state.pyr is not None and len(xy):
            r = temporal(state.pyr[c], pyrs[c], xy, p, net, n_threads)
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
