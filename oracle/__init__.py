"""CPU oracle of the VkVIO stereo frontend (arxiv 2609.30459, Sec. III).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the product library
never imports, loads or calls it. It shares no code with the CUDA path: the C++
sources under ``oracle/src`` restate the paper on their own, in integer
arithmetic where the paper fixes it and FP64 elsewhere.

Functions and the passage each follows:

* ``pyr_down`` / ``pyramid``     -- Sec. III-C, Eq. 1 (the 2-D double sum).
* ``fast_scores`` / ``fast_ring`` -- Sec. III-D, FAST-9 segment test and score.
* ``detect_grid``                -- Sec. III-D, threshold sequence, 3x3 NMS and
                                    per-cell top-k (literal loop, or one pass).
* ``pattern``                    -- Sec. III-E, the 52-point sample pattern
                                    (the offsets are this oracle's reading).
* ``template`` / ``se2_exp``     -- Sec. III-E, J, H, G and Eq. 5's exponential.
* ``track``                      -- Sec. III-E, Eq. 4-5, pyramidal IC-KLT with
                                    the forward-backward check.
* ``frontend.step``              -- Sec. III-B, the per-frame stage order.
* ``predict.predict_warp``       -- Sec. III-E, the start of a track from the
                                    camera model, predicted pose and inverse
                                    depth.

Parity unpinned (definitions the paper leaves open, pinned only by the GPU
matching this oracle): the pattern offsets, the bounds and degeneracy rules,
the forward-backward threshold value and the per-cell tie-break.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "src")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["pyramid_detect.cpp", "klt.cpp"]
_lock = threading.Lock()
_lib = None

STATUS = {
    "OK": 0,
    "OOB_TEMPLATE": 1,
    "OOB_WARP": 2,
    "DEGENERATE_H": 3,
    "ZERO_MEAN": 4,
    "FB_FAIL": 5,
    "NAN": 6,
}

# Paper constants (Sec. III-D, III-E, IV-D).
THRESHOLDS = (40, 20, 10, 5)
GN_ITERS = 5


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (portable flags; no -march, no fast-math)."""
    srcs = [os.path.join(_SRC, s) for s in _SOURCES]
    deps = srcs + [os.path.join(_SRC, "oracle.h")]
    if not force and os.path.exists(_LIB_PATH):
        lib_t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(d) <= lib_t for d in deps):
            return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Image(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("w", ctypes.c_int32),
                ("h", ctypes.c_int32), ("pitch", ctypes.c_int32)]


class _Pyramid(ctypes.Structure):
    _fields_ = [("lv", _Image * 8), ("n_levels", ctypes.c_int32)]


class _DetectParams(ctypes.Structure):
    _fields_ = [("cell_w", ctypes.c_int32), ("cell_h", ctypes.c_int32),
                ("k", ctypes.c_int32), ("n_thresholds", ctypes.c_int32),
                ("thresholds", ctypes.c_int32 * 8), ("border", ctypes.c_int32)]


class _TrackParams(ctypes.Structure):
    _fields_ = [("gn_iters", ctypes.c_int32), ("pattern_id", ctypes.c_int32),
                ("fb_max_dist", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32 = ctypes.c_int32
            lib.vo_pyr_down.argtypes = [P, i32, i32, i32, P, i32, i32]
            lib.vo_fast_scores.argtypes = [P, i32, i32, i32, P]
            lib.vo_fast_ring.argtypes = [P, P]
            lib.vo_detect_grid.argtypes = [P, i32, i32, i32, ctypes.POINTER(_DetectParams),
                                           P, P, i32, P, P, i32, i32]
            lib.vo_detect_grid.restype = i32
            lib.vo_pattern.argtypes = [i32, P, P]
            lib.vo_pattern.restype = i32
            lib.vo_track.argtypes = [ctypes.POINTER(_Pyramid), ctypes.POINTER(_Pyramid), i32,
                                     P, P, ctypes.POINTER(_TrackParams), i32, P, P, P, P, P,
                                     P, i32]
            lib.vo_template.argtypes = [ctypes.POINTER(_Image), ctypes.c_double,
                                        ctypes.c_double, i32, P, P, P, P, P, P, P]
            lib.vo_template.restype = i32
            lib.vo_se2_exp.argtypes = [ctypes.c_double] * 3 + [P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _u8(img) -> np.ndarray:
    a = np.ascontiguousarray(img)
    if a.dtype != np.uint8 or a.ndim != 2:
        raise ValueError("expected a 2-D uint8 image")
    return a


def pyr_down(img: np.ndarray, round_mode: int = 0) -> np.ndarray:
    """Eq. 1: the next pyramid level, floor(w/2) x floor(h/2)."""
    lib = _load()
    a = _u8(img)
    h, w = a.shape
    out = np.zeros((h // 2, w // 2), np.uint8)
    lib.vo_pyr_down(_ptr(a), w, h, w, _ptr(out), max(w // 2, 1), round_mode)
    return out


def pyramid(img: np.ndarray, n_levels: int, round_mode: int = 0) -> list[np.ndarray]:
    """Levels L0..L_{n-1} (Sec. III-C)."""
    levels = [_u8(img)]
    for _ in range(n_levels - 1):
        levels.append(pyr_down(levels[-1], round_mode))
    return levels


def fast_ring() -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    dx = np.zeros(16, np.int32)
    dy = np.zeros(16, np.int32)
    lib.vo_fast_ring(_ptr(dx), _ptr(dy))
    return dx, dy


def fast_scores(img: np.ndarray) -> np.ndarray:
    """FAST-9 score per pixel; -1 = not a corner (Sec. III-D)."""
    lib = _load()
    a = _u8(img)
    h, w = a.shape
    out = np.zeros((h, w), np.int16)
    lib.vo_fast_scores(_ptr(a), w, h, w, _ptr(out))
    return out


def detect_grid(img, cell_w, cell_h, k=1, thresholds=THRESHOLDS, border=9, occupancy=None,
                mask=None, one_pass=False, capacity=None):
    """Grid-cell detection (Sec. III-D). Returns (kp float32 (n,2), score int16 (n,))."""
    lib = _load()
    a = _u8(img)
    h, w = a.shape
    p = _DetectParams()
    p.cell_w, p.cell_h, p.k = cell_w, cell_h, k
    p.n_thresholds = len(thresholds)
    for i, t in enumerate(thresholds):
        p.thresholds[i] = int(t)
    p.border = border
    gx, gy = w // cell_w, h // cell_h
    if capacity is None:
        capacity = max(gx * gy * k, 1)
    occ = None if occupancy is None else np.ascontiguousarray(occupancy, np.uint8).reshape(-1)
    if occ is not None and occ.size != gx * gy:
        raise ValueError("occupancy must have one entry per cell")
    m = None if mask is None else _u8(mask)
    kp = np.zeros((capacity, 2), np.float32)
    sc = np.zeros(capacity, np.int16)
    n = lib.vo_detect_grid(_ptr(a), w, h, w, ctypes.byref(p), _ptr(occ), _ptr(m),
                           0 if m is None else m.shape[1], _ptr(kp), _ptr(sc), capacity,
                           1 if one_pass else 0)
    return kp[:n].copy(), sc[:n].copy()


def pattern(pattern_id: int = 0) -> np.ndarray:
    """Sample offsets (n, 2) of a pattern (Sec. III-E)."""
    lib = _load()
    u = np.zeros(64)
    v = np.zeros(64)
    n = lib.vo_pattern(pattern_id, _ptr(u), _ptr(v))
    return np.stack([u[:n], v[:n]], axis=1)


def _pyr_struct(levels: list[np.ndarray]):
    p = _Pyramid()
    keep = []
    for i, lv in enumerate(levels):
        a = _u8(lv)
        keep.append(a)
        p.lv[i].data = a.ctypes.data
        p.lv[i].h, p.lv[i].w = a.shape
        p.lv[i].pitch = a.shape[1]
    p.n_levels = len(levels)
    return p, keep


def track(src_levels, dst_levels, pts, init=None, gn_iters=GN_ITERS, pattern_id=0, fb=True,
          fb_max_dist=0.2, n_threads=1):
    """Pyramidal IC-KLT, optionally with the forward-backward check (Sec. III-E).

    Returns a dict with ``warp`` (n,3) float64 forward result (tx, ty, theta)
    in level-0 px, ``status`` (n,) uint8, ``fb_dist`` (n,) float64, ``margin``
    (n,) float64, ``back`` (n,3) float64 and ``last_step`` (n,) float64 (the
    forward pass's last level-0 step, |dx| + |dy| + r |dtheta|)."""
    lib = _load()
    pts = np.ascontiguousarray(pts, np.float32).reshape(-1, 2)
    n = pts.shape[0]
    ini = None if init is None else np.ascontiguousarray(init, np.float32).reshape(-1, 3)
    sp, k1 = _pyr_struct(src_levels)
    dp, k2 = _pyr_struct(dst_levels)
    prm = _TrackParams()
    prm.gn_iters, prm.pattern_id, prm.fb_max_dist = gn_iters, pattern_id, fb_max_dist
    warp = np.zeros((n, 3))
    status = np.zeros(n, np.uint8)
    fbd = np.zeros(n)
    margin = np.zeros(n)
    back = np.zeros((n, 3))
    last = np.zeros(n)
    lib.vo_track(ctypes.byref(sp), ctypes.byref(dp), n, _ptr(pts), _ptr(ini), ctypes.byref(prm),
                 1 if fb else 0, _ptr(warp), _ptr(status), _ptr(fbd), _ptr(margin), _ptr(back),
                 _ptr(last), n_threads)
    del k1, k2
    return {"warp": warp, "status": status, "fb_dist": fbd, "margin": margin, "back": back,
            "last_step": last}


def template(img, qx, qy, pattern_id=0):
    """Template quantities at one level (Sec. III-E): dict of s, gx, gy, J, H, G, mean, status."""
    lib = _load()
    a = _u8(img)
    im = _Image()
    im.data = a.ctypes.data
    im.h, im.w = a.shape
    im.pitch = a.shape[1]
    n = len(pattern(pattern_id))
    s, gx, gy = np.zeros(n), np.zeros(n), np.zeros(n)
    J = np.zeros((n, 3))
    H = np.zeros((3, 3))
    G = np.zeros((3, n))
    mean = ctypes.c_double(0)
    st = lib.vo_template(ctypes.byref(im), qx, qy, pattern_id, _ptr(s), _ptr(gx), _ptr(gy),
                         _ptr(J), _ptr(H), _ptr(G), ctypes.cast(ctypes.pointer(mean),
                                                                ctypes.c_void_p))
    return {"status": st, "s": s, "gx": gx, "gy": gy, "J": J, "H": H, "G": G,
            "mean": mean.value}


def se2_exp(dx, dy, dth) -> np.ndarray:
    """Eq. 5's exponential map as a 3x3 homogeneous matrix."""
    lib = _load()
    M = np.zeros(9)
    lib.vo_se2_exp(dx, dy, dth, _ptr(M))
    return M.reshape(3, 3)
