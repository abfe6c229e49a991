"""Thin ctypes binding of libvio (include/vio.h): argument marshalling only.

Every function here takes torch CUDA tensors, passes their device pointers and
the current CUDA stream to the C ABI, and returns. All computation happens in
the library's kernels. There is no CPU fallback: if libvio.so is missing or no
GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build_lib

MAX_LEVELS = 8
MAX_THRESHOLDS = 8

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_UNSUPPORTED = range(6)
TRACK_STATUS = {"OK": 0, "OOB_TEMPLATE": 1, "OOB_WARP": 2, "DEGENERATE_H": 3, "ZERO_MEAN": 4,
                "FB_FAIL": 5, "NAN": 6, "EMPTY": 255}
TRACK_FORWARD, TRACK_WITH_FB = 0, 1


class Params(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int32), ("round_mode", ctypes.c_int32),
                ("gn_iters", ctypes.c_int32), ("pattern_id", ctypes.c_int32),
                ("cell_w", ctypes.c_int32), ("cell_h", ctypes.c_int32),
                ("k_per_cell", ctypes.c_int32), ("n_thresholds", ctypes.c_int32),
                ("thresholds", ctypes.c_int32 * MAX_THRESHOLDS),
                ("detect_border", ctypes.c_int32), ("fb_max_dist", ctypes.c_float),
                ("select_mode", ctypes.c_int32)]


class PyrLayout(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int32), ("w", ctypes.c_int32 * MAX_LEVELS),
                ("h", ctypes.c_int32 * MAX_LEVELS), ("pitch", ctypes.c_int32 * MAX_LEVELS),
                ("offset", ctypes.c_int64 * MAX_LEVELS), ("upper_bytes", ctypes.c_int64)]


class PyrBatch(ctypes.Structure):
    _fields_ = [("d_level0", ctypes.c_void_p), ("level0_stride", ctypes.c_int64),
                ("d_upper", ctypes.c_void_p), ("upper_stride", ctypes.c_int64),
                ("n_images", ctypes.c_int32)]


class FrontendView(ctypes.Structure):
    _fields_ = [("d_track_xy", ctypes.c_void_p), ("d_track_id", ctypes.c_void_p),
                ("d_track_status", ctypes.c_void_p), ("d_track_count", ctypes.c_void_p),
                ("d_new_xy", ctypes.c_void_p), ("d_new_count", ctypes.c_void_p),
                ("capacity", ctypes.c_int32), ("n_streams", ctypes.c_int32)]


class StreamGroup(ctypes.Structure):
    _fields_ = [("params", Params), ("w", ctypes.c_int32), ("h", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("capacity", ctypes.c_int32)]


class BatchTune(ctypes.Structure):
    _fields_ = [("k2_threads", ctypes.c_int32), ("pyr_tile_shift", ctypes.c_int32),
                ("stereo_after_select", ctypes.c_int32), ("pyr_first_levels", ctypes.c_int32),
                ("k1_threads", ctypes.c_int32),
                ("det_warps", ctypes.c_int32)]


class Pinhole(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float)]


class InitNetCfg(ctypes.Structure):
    _fields_ = [("level_a", ctypes.c_int32), ("level_b", ctypes.c_int32),
                ("start_level", ctypes.c_int32), ("min_conf", ctypes.c_float),
                ("max_last_step", ctypes.c_float)]


class ServerReq(ctypes.Structure):
    _fields_ = [("session", ctypes.c_int64), ("t_offset", ctypes.c_double),
                ("host_frame", ctypes.c_void_p), ("tag", ctypes.c_int64),
                ("flags", ctypes.c_int32)]


class ServerDone(ctypes.Structure):
    _fields_ = [("session", ctypes.c_int64), ("tag", ctypes.c_int64),
                ("t_arrival", ctypes.c_double), ("t_launch", ctypes.c_double),
                ("t_done", ctypes.c_double), ("n_tracks", ctypes.c_int32 * 2),
                ("n_new", ctypes.c_int32), ("status", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()

_SIGS = {
    "vio_params_default": (None, [ctypes.POINTER(Params)]),
    "vio_status_string": (ctypes.c_char_p, [ctypes.c_int32]),
    "vio_pyr_layout_make": (ctypes.c_int32, [ctypes.c_int32] * 4 + [ctypes.POINTER(PyrLayout)]),
    "vio_ctx_create": (ctypes.c_int32, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Params),
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "vio_ctx_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "vio_ctx_sync": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_int32)]),
    "vio_last_error": (ctypes.c_int32, [ctypes.c_void_p]),
    "vio_wait_flag": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_int64, ctypes.c_void_p]),
    "vio_pyramid_build": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(PyrLayout),
                                           ctypes.POINTER(PyrBatch), ctypes.c_void_p]),
    "vio_fast_scores": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "vio_detect_grid": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(PyrLayout),
                                         ctypes.POINTER(PyrBatch), ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_void_p]),
    "vio_pyramid_detect": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(PyrLayout),
                                            ctypes.POINTER(PyrBatch), ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_void_p]),
    "vio_detect_grid_noalloc": (ctypes.c_int32, [ctypes.POINTER(Params), ctypes.POINTER(PyrLayout),
                                                 ctypes.POINTER(PyrBatch), ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_int64,
                                                 ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_int32,
                                                 ctypes.c_void_p]),
    "vio_track_patches": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(PyrLayout),
                                           ctypes.POINTER(PyrBatch), ctypes.POINTER(PyrBatch),
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "vio_stereo_match": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(PyrLayout),
                                          ctypes.POINTER(PyrBatch), ctypes.POINTER(PyrBatch),
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "vio_predict_warp": (ctypes.c_int32, [ctypes.POINTER(Pinhole), ctypes.POINTER(Pinhole),
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vio_match_cameras": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(PyrLayout),
                                           ctypes.POINTER(PyrBatch), ctypes.POINTER(PyrBatch),
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "vio_fb_check": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vio_frontend_create": (ctypes.c_int32, [ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.POINTER(Params), ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "vio_frontend_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "vio_frontend_step": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_int64, ctypes.c_void_p]),
    "vio_frontend_reset": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p]),
    "vio_frontend_step_host": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_int32,
                                                ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]),
    "vio_frontend_step_host_async": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_int32,
                                                ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]),
    "vio_frontend_get_view": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(FrontendView)]),
    "vio_frontend_launches_per_step": (ctypes.c_int32, [ctypes.c_void_p]),
    "vio_frontend_set_tune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(BatchTune)]),
    "vio_frontend_set_timing": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "vio_frontend_read_timing": (ctypes.c_int32, [ctypes.c_void_p,
                                                  ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_int64),
                                                  ctypes.c_void_p, ctypes.c_int64]),
    "vio_frontend_run": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_void_p]),
    "vio_frontend_read_stats": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.POINTER(ctypes.c_int64)]),
    "vio_batch_create": (ctypes.c_int32, [ctypes.POINTER(ctypes.c_void_p),
                                          ctypes.POINTER(StreamGroup), ctypes.c_int32]),
    "vio_batch_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "vio_batch_next_frame": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_void_p)]),
    "vio_batch_step": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vio_batch_set_graph": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "vio_batch_set_tune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(BatchTune)]),
    "vio_batch_get_tune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(BatchTune)]),
    "vio_batch_autotune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_float)]),
    "vio_batch_reset_stream": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_void_p]),
    "vio_batch_get_view": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.POINTER(FrontendView), ctypes.c_void_p]),
    "vio_batch_launches_per_step": (ctypes.c_int32, [ctypes.c_void_p]),
    "vio_batch_read_stats": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                              ctypes.POINTER(ctypes.c_int64)]),
    "vio_frontend_set_initnet": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.POINTER(InitNetCfg)]),
    "vio_batch_set_initnet": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.POINTER(InitNetCfg)]),
    "vio_batch_device_bytes": (ctypes.c_int32, [ctypes.POINTER(StreamGroup), ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_int64)]),
    "vio_server_now": (ctypes.c_double, []),
    "vio_server_plan": (ctypes.c_int32, [ctypes.POINTER(StreamGroup), ctypes.c_int32,
                                         ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_int64)]),
    "vio_server_create": (ctypes.c_int32, [ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(StreamGroup), ctypes.c_int32,
                                           ctypes.c_int64]),
    "vio_server_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "vio_server_slots": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int64)]),
    "vio_server_set_initnet": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.POINTER(InitNetCfg)]),
    "vio_server_set_tune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(BatchTune)]),
    "vio_server_open": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int32)]),
    "vio_server_set_output": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]),
    "vio_server_submit": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_double, ctypes.c_int64, ctypes.c_int32]),
    "vio_server_close": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int64]),
    "vio_server_poll": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "vio_server_take": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ServerDone),
                                         ctypes.c_int32]),
    "vio_server_run_trace": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ServerReq),
                                              ctypes.c_int64, ctypes.POINTER(ServerDone),
                                              ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]),
    "vio_server_set_loop_policy": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32,
                                                    ctypes.c_int32]),
    "vio_server_loop_policy_granted": (ctypes.c_int32, [ctypes.c_void_p,
                                                        ctypes.POINTER(ctypes.c_int32)]),
    "vio_server_loop_stats": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_int64)]),
    "vio_initnet_pack": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vio_initnet_extract": (ctypes.c_int32, [ctypes.POINTER(PyrLayout), ctypes.POINTER(PyrBatch),
                                             ctypes.POINTER(PyrBatch), ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "vio_initnet_forward": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                             ctypes.c_void_p, ctypes.c_void_p]),
    "vio_initnet_fault": (ctypes.c_int32, [ctypes.POINTER(ctypes.c_int32)]),
    "vio_initnet_train_step": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                                ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]),
    "vio_initnet_adam": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int32, ctypes.c_float,
                                          ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                          ctypes.c_void_p]),
}

STAGES = ("front", "pyramid_upper", "initnet", "track", "finalize")
STATS_RING = 4096
STAT_NAMES = ("trk0", "trk1", "ok0", "ok1", "new", "matched", "cand", "learned")


def lib_path() -> str:
    return build_lib.LIB


def load(build: bool = False) -> ctypes.CDLL:
    """Load libvio.so (building it first if asked). Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if build:
                build_lib.build()
            if not os.path.exists(build_lib.LIB):
                raise RuntimeError(f"libvio.so not built ({build_lib.LIB}); run "
                                   "__graft_entry__.build() or build_lib.build()")
            lib = ctypes.CDLL(build_lib.LIB)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


class VioError(RuntimeError):
    pass


def _check(status: int, what: str):
    if status != OK:
        msg = load().vio_status_string(status).decode()
        raise VioError(f"{what} failed: {msg} ({status})")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def default_params(**kw) -> Params:
    p = Params()
    load().vio_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if k == "thresholds":
            p.n_thresholds = len(v)
            for i, t in enumerate(v):
                p.thresholds[i] = int(t)
        else:
            setattr(p, k, v)
    return p


def pyr_layout(w: int, h: int, n_levels: int, level0_pitch: int | None = None) -> PyrLayout:
    L = PyrLayout()
    _check(load().vio_pyr_layout_make(w, h, n_levels, level0_pitch or w, ctypes.byref(L)),
           "vio_pyr_layout_make")
    return L


class Pyramids:
    """n images of one size and their upper pyramid levels, on the device.

    level0: uint8 tensor (n, h, pitch) holding level 0 (the frames)."""

    def __init__(self, level0: torch.Tensor, n_levels: int, w: int | None = None):
        if level0.dtype != torch.uint8 or level0.dim() != 3 or not level0.is_cuda:
            raise ValueError("level0 must be a CUDA uint8 tensor (n, h, pitch)")
        n, h, pitch = level0.shape
        self.level0 = level0.contiguous()
        self.w = w or pitch
        self.h = h
        self.n = n
        self.layout = pyr_layout(self.w, h, n_levels, pitch)
        ub = int(self.layout.upper_bytes)
        self.upper = torch.empty(max(n * ub, 16), dtype=torch.uint8, device=level0.device)

    def batch(self, start: int = 0, step: int = 1, count: int | None = None) -> PyrBatch:
        count = count if count is not None else (self.n - start + step - 1) // step
        b = PyrBatch()
        ub = int(self.layout.upper_bytes)
        b.d_level0 = self.level0.data_ptr() + start * self.level0[0].numel()
        b.level0_stride = step * self.level0[0].numel()
        b.d_upper = self.upper.data_ptr() + start * ub
        b.upper_stride = step * ub
        b.n_images = count
        return b

    def level(self, i: int, l: int) -> torch.Tensor:
        """View of level l of image i as (h_l, w_l) uint8 (device)."""
        L = self.layout
        if l == 0:
            return self.level0[i, :, : self.w]
        ub = int(L.upper_bytes)
        off = i * ub + int(L.offset[l])
        flat = self.upper[off: off + L.pitch[l] * L.h[l]]
        return flat.view(L.h[l], L.pitch[l])[:, : L.w[l]]


class Context:
    """vio_ctx: parameters plus the scratch the detection stage needs."""

    def __init__(self, params: Params, max_w: int, max_h: int, max_images: int):
        self.params = params
        h = ctypes.c_void_p()
        _check(load().vio_ctx_create(ctypes.byref(h), ctypes.byref(params), max_w, max_h,
                                     max_images), "vio_ctx_create")
        self.handle = h

    def close(self):
        if self.handle:
            load().vio_ctx_destroy(self.handle)
            self.handle = None

    def sync(self, stream=None) -> int:
        """vio_ctx_sync: waits for the stream, returns and clears the device
        status word (OK, or e.g. ERR_TIMEOUT from a bounded wait)."""
        st = ctypes.c_int32()
        _check(load().vio_ctx_sync(self.handle, _stream(stream), ctypes.byref(st)),
               "vio_ctx_sync")
        return int(st.value)

    def last_error(self) -> int:
        """vio_last_error: the device status word, not cleared."""
        return int(load().vio_last_error(self.handle))

    def wait_flag(self, flag, value: int, timeout_ns: int, stream=None):
        """vio_wait_flag: the stream waits until the int32 flag (CUDA tensor)
        equals value, for at most timeout_ns."""
        _check(load().vio_wait_flag(self.handle, _ptr(flag), int(value), int(timeout_ns),
                                    _stream(stream)), "vio_wait_flag")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- stages --------------------------------------------------------------
    def pyramid_build(self, pyr: Pyramids, batch: PyrBatch | None = None, stream=None):
        _check(load().vio_pyramid_build(self.handle, ctypes.byref(pyr.layout),
                                        ctypes.byref(batch or pyr.batch()), _stream(stream)),
               "vio_pyramid_build")

    def detect_grid(self, pyr: Pyramids, batch: PyrBatch, kp, score, count, capacity,
                    occupancy=None, mask=None, mask_stride=0, stream=None):
        _check(load().vio_detect_grid(self.handle, ctypes.byref(pyr.layout), ctypes.byref(batch),
                                      _ptr(occupancy), _ptr(mask), mask_stride, _ptr(kp),
                                      _ptr(score), _ptr(count), capacity, _stream(stream)),
               "vio_detect_grid")

    def pyramid_detect(self, pyr: Pyramids, kp, score, count, capacity, occupancy=None,
                       mask=None, mask_stride=0, batch: PyrBatch | None = None, stream=None):
        """Pyramid and detection of every image of the batch, fused."""
        _check(load().vio_pyramid_detect(self.handle, ctypes.byref(pyr.layout),
                                         ctypes.byref(batch or pyr.batch()), _ptr(occupancy),
                                         _ptr(mask), mask_stride, _ptr(kp), _ptr(score),
                                         _ptr(count), capacity, _stream(stream)),
               "vio_pyramid_detect")

    def track_patches(self, pyr: Pyramids, src: PyrBatch, dst: PyrBatch, pts, count, capacity,
                      out, status, fb_dist=None, init=None, fb=True, from_level=None,
                      last_step=None, stream=None):
        """from_level: track over levels from_level..0 only (default: all);
        last_step: per keypoint, the forward pass's last level-0 step size."""
        flags = TRACK_WITH_FB if fb else TRACK_FORWARD
        if from_level is not None:
            flags |= (int(from_level) + 1) << 4
        _check(load().vio_track_patches(self.handle, ctypes.byref(pyr.layout), ctypes.byref(src),
                                        ctypes.byref(dst), _ptr(pts), _ptr(init), _ptr(count),
                                        capacity, flags, _ptr(out), _ptr(status), _ptr(fb_dist),
                                        _ptr(last_step), _stream(stream)), "vio_track_patches")

    def match_cameras(self, pyr: Pyramids, src: PyrBatch, dst: PyrBatch, pts, count, capacity,
                      match, status, fb_dist=None, init=None, stream=None):
        """vio_match_cameras: the keypoints of the one source image tracked (with
        the FB check) into every target image of dst."""
        _check(load().vio_match_cameras(self.handle, ctypes.byref(pyr.layout), ctypes.byref(src),
                                        ctypes.byref(dst), _ptr(pts), _ptr(init), _ptr(count),
                                        capacity, _ptr(match), _ptr(status), _ptr(fb_dist),
                                        _stream(stream)), "vio_match_cameras")

    def stereo_match(self, pyr: Pyramids, cam0: PyrBatch, cam1: PyrBatch, pts, count, capacity,
                     match, status, fb_dist=None, init=None, stream=None):
        _check(load().vio_stereo_match(self.handle, ctypes.byref(pyr.layout), ctypes.byref(cam0),
                                       ctypes.byref(cam1), _ptr(pts), _ptr(init), _ptr(count),
                                       capacity, _ptr(match), _ptr(status), _ptr(fb_dist),
                                       _stream(stream)), "vio_stereo_match")


def fast_scores(img: torch.Tensor, out: torch.Tensor | None = None, w: int | None = None,
                stream=None) -> torch.Tensor:
    """FAST-9 score map of one uint8 image (h, pitch) -> int16 (h, w)."""
    h, pitch = img.shape
    w = w or pitch
    if out is None:
        out = torch.empty((h, w), dtype=torch.int16, device=img.device)
    _check(load().vio_fast_scores(_ptr(img), w, h, pitch, _ptr(out), _stream(stream)),
           "vio_fast_scores")
    return out


NOALLOC_MAX_CELL_SLOTS = 65536


def detect_grid_noalloc(params: Params, pyr: "Pyramids", batch: PyrBatch, kp, score, count,
                        capacity, occupancy=None, mask=None, mask_stride=0, stream=None):
    """vio_detect_grid_noalloc: detection for callers that cannot allocate
    device memory (no vio_ctx; the scratch is a fixed array inside the library,
    shared by all calls, so calls must not overlap on the GPU)."""
    _check(load().vio_detect_grid_noalloc(ctypes.byref(params), ctypes.byref(pyr.layout),
                                          ctypes.byref(batch), _ptr(occupancy), _ptr(mask),
                                          mask_stride, _ptr(kp), _ptr(score), _ptr(count),
                                          capacity, _stream(stream)),
           "vio_detect_grid_noalloc")


def predict_warp(k_src, k_dst, poses, pts, inv_depth, count, capacity, n_images, init,
                 valid=None, stream=None):
    """vio_predict_warp: the model-based start of each keypoint's warp.
    k_src, k_dst: (fx, fy, cx, cy); poses: float32 CUDA tensor (n_images, 12),
    each row R (row-major, 9) then t (3), mapping source-camera points into the
    target camera; pts (n_images, capacity, 2), inv_depth (n_images, capacity),
    init (n_images, capacity, 3) float32, valid (n_images, capacity) uint8."""
    ks, kd = Pinhole(*[float(v) for v in k_src]), Pinhole(*[float(v) for v in k_dst])
    _check(load().vio_predict_warp(ctypes.byref(ks), ctypes.byref(kd), _ptr(poses), _ptr(pts),
                                   _ptr(inv_depth), _ptr(count), capacity, n_images, _ptr(init),
                                   _ptr(valid), _stream(stream)), "vio_predict_warp")


def fb_check(orig, back, count, capacity, n_images, max_dist, status, dist=None, stream=None):
    _check(load().vio_fb_check(_ptr(orig), _ptr(back), _ptr(count), capacity, n_images,
                               max_dist, _ptr(status), _ptr(dist), _stream(stream)),
           "vio_fb_check")


INITNET_N_PARAMS = 28131
INITNET_PACKED_BYTES = 58016


def initnet_pack(master, packed, stream=None):
    """FP32 master parameters (INITNET_N_PARAMS) -> packed BF16 weights."""
    _check(load().vio_initnet_pack(_ptr(master), _ptr(packed), _stream(stream)),
           "vio_initnet_pack")


def initnet_extract(pyr: Pyramids, src: PyrBatch, dst: PyrBatch, pts, count, capacity,
                    level_a, level_b, x, stream=None):
    """Network inputs (bf16 bits as int16, [n][4][16][16]) of keypoints."""
    _check(load().vio_initnet_extract(ctypes.byref(pyr.layout), ctypes.byref(src),
                                      ctypes.byref(dst), _ptr(pts), _ptr(count), capacity,
                                      level_a, level_b, _ptr(x), _stream(stream)),
           "vio_initnet_extract")


def initnet_forward(packed, x, n, out, stream=None):
    _check(load().vio_initnet_forward(_ptr(packed), _ptr(x), n, _ptr(out), _stream(stream)),
           "vio_initnet_forward")


def initnet_fault() -> int:
    """vio_initnet_fault: the tensor-core forward passes' status word (VIO_OK
    or VIO_ERR_TIMEOUT), read and cleared."""
    v = ctypes.c_int32(0)
    _check(load().vio_initnet_fault(ctypes.byref(v)), "vio_initnet_fault")
    return int(v.value)


def initnet_train_step(packed, x, flow, index, n, grad_scale, grad, loss, label_radius=1.0,
                       stream=None):
    _check(load().vio_initnet_train_step(_ptr(packed), _ptr(x), _ptr(flow), _ptr(index), n,
                                         grad_scale, label_radius, _ptr(grad), _ptr(loss),
                                         _stream(stream)), "vio_initnet_train_step")


def initnet_adam(master, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().vio_initnet_adam(_ptr(master), _ptr(grad), _ptr(m), _ptr(v), step, lr, beta1,
                                   beta2, eps, _stream(stream)), "vio_initnet_adam")


class InitNet:
    """Learned flow initializer on the device: FP32 master parameters, their
    packed BF16 copy (what the kernels read) and the gate configuration.

    Checkpoints are .npz files holding ``master`` (and, for resuming
    training, the Adam moments ``m``, ``v`` and the step count) plus the
    configuration; no pickled objects."""

    # a learned track counts only if its last level-0 step moved the pattern
    # by at most this (px); the plain track otherwise
    DEFAULT_MAX_LAST_STEP = 1e-3

    def __init__(self, master=None, level_a=2, level_b=3, start_level=1, min_conf=0.5,
                 device="cuda", max_last_step=DEFAULT_MAX_LAST_STEP):
        if master is None:
            master = torch.zeros(INITNET_N_PARAMS, dtype=torch.float32)
        master = torch.as_tensor(master, dtype=torch.float32).reshape(-1)
        if master.numel() != INITNET_N_PARAMS:
            raise ValueError(f"expected {INITNET_N_PARAMS} parameters, got {master.numel()}")
        self.master = master.to(device).contiguous()
        self.packed = torch.empty(INITNET_PACKED_BYTES, dtype=torch.uint8, device=device)
        self.cfg = InitNetCfg(level_a, level_b, start_level, min_conf, max_last_step)
        self.m = None
        self.v = None
        self.step = 0
        self.pack()

    def pack(self, stream=None):
        initnet_pack(self.master, self.packed, stream)

    def configure(self, **kw):
        for k, v in kw.items():
            setattr(self.cfg, k, v)

    def forward(self, x, out=None, stream=None):
        """x: int16 CUDA tensor (n, 4, 16, 16) of BF16 bits -> (n, 3) dx, dy, conf."""
        n = x.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32, device=x.device)
        initnet_forward(self.packed, x, n, out, stream)
        return out

    def save(self, path, **meta):
        """meta: further named values stored beside the weights (numbers)."""
        import numpy as np
        extra = {k: np.asarray(v) for k, v in meta.items()}
        if self.m is not None:
            extra.update(m=self.m.cpu().numpy(), v=self.v.cpu().numpy())
        np.savez(path, master=self.master.cpu().numpy(),
                 cfg=np.array([self.cfg.level_a, self.cfg.level_b, self.cfg.start_level],
                              np.int32),
                 min_conf=np.array([self.cfg.min_conf], np.float32),
                 max_last_step=np.array([self.cfg.max_last_step], np.float32),
                 step=np.array([self.step], np.int64), **extra)

    @classmethod
    def load(cls, path, device="cuda"):
        import numpy as np
        with np.load(path, allow_pickle=False) as z:
            cfg = z["cfg"]
            net = cls(z["master"], int(cfg[0]), int(cfg[1]), int(cfg[2]),
                      float(z["min_conf"][0]), device,
                      float(z["max_last_step"][0]) if "max_last_step" in z
                      else cls.DEFAULT_MAX_LAST_STEP)
            net.step = int(z["step"][0])
            if "m" in z:
                net.m = torch.from_numpy(z["m"]).to(device)
                net.v = torch.from_numpy(z["v"]).to(device)
        return net


class Frontend:
    """vio_frontend: the per-frame frontend over n_streams stereo streams."""

    def __init__(self, params: Params, w: int, h: int, n_streams: int, capacity: int):
        self.params, self.w, self.h = params, w, h
        self.n_streams, self.capacity = n_streams, capacity
        hdl = ctypes.c_void_p()
        _check(load().vio_frontend_create(ctypes.byref(hdl), ctypes.byref(params), w, h,
                                          n_streams, capacity), "vio_frontend_create")
        self.handle = hdl

    def close(self):
        if self.handle:
            load().vio_frontend_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, frames: torch.Tensor, stream=None):
        """frames: uint8 CUDA tensor (n_streams, 2, h, pitch); kept alive by the
        caller until the next step has run."""
        if frames.dtype != torch.uint8 or frames.dim() != 4 or not frames.is_contiguous():
            raise ValueError("frames must be a contiguous uint8 tensor (streams, 2, h, pitch)")
        pitch = frames.shape[-1]
        _check(load().vio_frontend_step(self.handle, _ptr(frames), pitch,
                                        frames.shape[2] * pitch, _stream(stream)),
               "vio_frontend_step")

    def reset(self, stream=None):
        _check(load().vio_frontend_reset(self.handle, _stream(stream)), "vio_frontend_reset")

    def host_outputs(self):
        """Pinned host buffers for step_host: dict of xy, id, count, new_xy, new_count."""
        ns, cap = self.n_streams, self.capacity
        pin = dict(dtype=torch.float32, pin_memory=True)
        return {"xy": torch.empty((ns, 2, cap, 2), **pin),
                "id": torch.empty((ns, 2, cap), dtype=torch.int32, pin_memory=True),
                "count": torch.empty((ns, 2), dtype=torch.int32, pin_memory=True),
                "new_xy": torch.empty((ns, cap, 2), **pin),
                "new_count": torch.empty((ns,), dtype=torch.int32, pin_memory=True)}

    def step_host(self, h_frames: torch.Tensor, d_frames: torch.Tensor, out: dict, stream=None):
        """One step from pinned host frames (streams, 2, h, pitch) through the
        device buffer d_frames (same shape, kept alive until the next step) to
        the pinned buffers of host_outputs(); asynchronous on the stream."""
        pitch = h_frames.shape[-1]
        _check(load().vio_frontend_step_host(self.handle, _hptr(h_frames), _ptr(d_frames), pitch,
                                             h_frames.shape[2] * pitch, _hptr(out["xy"]),
                                             _hptr(out["id"]), _hptr(out["count"]),
                                             _hptr(out["new_xy"]), _hptr(out["new_count"]),
                                             _stream(stream)), "vio_frontend_step_host")

    def step_host_async(self, h_frames: torch.Tensor, d_frames: torch.Tensor, out: dict,
                        done: "torch.cuda.Event | None" = None):
        """step_host pipelined across calls on the frontend's own streams; `done`
        (a recorded-once torch.cuda.Event) is recorded when `out` holds this
        step's results. d_frames must stay untouched until the next step's
        event."""
        pitch = h_frames.shape[-1]
        ev = ctypes.c_void_p(done.cuda_event) if done is not None else None
        _check(load().vio_frontend_step_host_async(
            self.handle, _hptr(h_frames), _ptr(d_frames), pitch, h_frames.shape[2] * pitch,
            _hptr(out["xy"]), _hptr(out["id"]), _hptr(out["count"]), _hptr(out["new_xy"]),
            _hptr(out["new_count"]), ev), "vio_frontend_step_host_async")

    def launches_per_step(self) -> int:
        return int(load().vio_frontend_launches_per_step(self.handle))

    def set_tune(self, k2_threads: int = 128, pyr_tile_shift: int = 0,
                 pyr_first_levels: int = 0, k1_threads: int = 256, det_warps: int = 0):
        t = BatchTune(k2_threads, pyr_tile_shift, 0, pyr_first_levels, k1_threads, det_warps)
        _check(load().vio_frontend_set_tune(self.handle, ctypes.byref(t)),
               "vio_frontend_set_tune")

    def set_initnet(self, net: "InitNet | None"):
        """Turn the learned start of temporal tracking on (net) or off (None).
        The frontend reads net.packed at every step: keep net alive."""
        self._net = net
        _check(load().vio_frontend_set_initnet(self.handle, _ptr(net.packed) if net else None,
                                               ctypes.byref(net.cfg) if net else None),
               "vio_frontend_set_initnet")

    def set_timing(self, enable):
        """False/0 off, True/1 events at every stage boundary, 2 only the first
        and last event of each step (vio_frontend_set_timing)."""
        _check(load().vio_frontend_set_timing(self.handle, int(enable)), "set_timing")

    def read_timing(self, max_steps: int = 0):
        """(summed per-stage ms, number of timed steps, per-step ms list) of the
        steps timed since the last read."""
        import numpy as np
        ms = (ctypes.c_double * len(STAGES))()
        n = ctypes.c_int64()
        steps = np.zeros(max(max_steps, 1), np.float32)
        _check(load().vio_frontend_read_timing(self.handle, ms, ctypes.byref(n),
                                               steps.ctypes.data_as(ctypes.c_void_p),
                                               max_steps), "read_timing")
        k = min(int(n.value), max_steps)
        return {s: ms[i] for i, s in enumerate(STAGES)}, int(n.value), steps[:k].tolist()

    def run(self, frames: torch.Tensor, stream=None):
        """Every frame of frames (n_steps, n_streams, 2, h, pitch), one step each,
        enqueued by one call."""
        if frames.dtype != torch.uint8 or frames.dim() != 5 or not frames.is_contiguous():
            raise ValueError("frames must be a contiguous uint8 tensor "
                             "(steps, streams, 2, h, pitch)")
        pitch = frames.shape[-1]
        fs = frames.shape[3] * pitch
        _check(load().vio_frontend_run(self.handle, _ptr(frames), pitch, fs, frames[0].numel(),
                                       frames.shape[0], _stream(stream)), "vio_frontend_run")

    def read_stats(self):
        """(ring array (STATS_RING, n_streams, 6) int32, steps run since create)."""
        import numpy as np
        out = np.zeros((STATS_RING, self.n_streams, len(STAT_NAMES)), np.int32)
        n = ctypes.c_int64()
        _check(load().vio_frontend_read_stats(self.handle, out.ctypes.data_as(ctypes.c_void_p),
                                              ctypes.byref(n)), "read_stats")
        return out, int(n.value)

    def view(self) -> dict:
        """Device tensors aliasing the frontend's outputs (no copies)."""
        v = FrontendView()
        _check(load().vio_frontend_get_view(self.handle, ctypes.byref(v)), "get_view")
        dev = torch.device("cuda", torch.cuda.current_device())
        ns, cap = self.n_streams, self.capacity
        return {
            "track_xy": _alias(v.d_track_xy, (ns, 2, cap, 2), torch.float32, dev),
            "track_id": _alias(v.d_track_id, (ns, 2, cap), torch.int32, dev),
            "track_status": _alias(v.d_track_status, (ns, 2, cap), torch.uint8, dev),
            "track_count": _alias(v.d_track_count, (ns, 2), torch.int32, dev),
            "new_xy": _alias(v.d_new_xy, (ns, cap, 2), torch.float32, dev),
            "new_count": _alias(v.d_new_count, (ns,), torch.int32, dev),
        }


def _alias(ptr: int, shape, dtype, device) -> torch.Tensor:
    """A tensor view of library-owned device memory (valid while the owner lives)."""
    n = 1
    for s in shape:
        n *= s
    nbytes = n * torch.empty((), dtype=dtype).element_size()

    class _Holder:
        __cuda_array_interface__ = {
            "shape": (nbytes,), "typestr": "|u1", "data": (int(ptr), False), "version": 3,
            "strides": None,
        }
    raw = torch.as_tensor(_Holder(), device=device)
    return raw.view(dtype).view(*shape)


class Batch:
    """vio_batch: stereo streams of mixed sizes stepped together (size groups).

    groups: list of (params, w, h, n_streams, capacity)."""

    def __init__(self, groups):
        arr = (StreamGroup * len(groups))()
        for i, (p, w, h, n, cap) in enumerate(groups):
            arr[i].params = p
            arr[i].w, arr[i].h, arr[i].n_streams, arr[i].capacity = w, h, n, cap
        self.groups = [(w, h, n, cap) for (_, w, h, n, cap) in groups]
        self.total = sum(g[2] for g in self.groups)
        hdl = ctypes.c_void_p()
        _check(load().vio_batch_create(ctypes.byref(hdl), arr, len(groups)), "vio_batch_create")
        self.handle = hdl

    def close(self):
        if self.handle:
            load().vio_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def next_frame(self, g: int, s: int) -> torch.Tensor:
        """Device view (2, h, w) uint8 of the slot stream s of group g reads next."""
        ptr = ctypes.c_void_p()
        _check(load().vio_batch_next_frame(self.handle, g, s, ctypes.byref(ptr)), "next_frame")
        w, h, _, _ = self.groups[g]
        dev = torch.device("cuda", torch.cuda.current_device())
        return _alias(ptr.value, (2, h, w), torch.uint8, dev)

    def step(self, active=None, stream=None):
        if active is None:
            arg = None
        else:
            import numpy as np
            a = np.ascontiguousarray(active, dtype=np.int32)
            if a.size != self.total:
                raise ValueError("one activity flag per stream")
            arg = a.ctypes.data_as(ctypes.c_void_p)
            self._keep = a
        _check(load().vio_batch_step(self.handle, arg, _stream(stream)), "vio_batch_step")

    def set_graph(self, enable: bool):
        _check(load().vio_batch_set_graph(self.handle, 1 if enable else 0), "set_graph")

    def set_tune(self, k2_threads: int, pyr_tile_shift: int, stereo_after_select: int = 0,
                 pyr_first_levels: int = 0, k1_threads: int = 256, det_warps: int = 0):
        t = BatchTune(k2_threads, pyr_tile_shift, stereo_after_select, pyr_first_levels,
                      k1_threads, det_warps)
        _check(load().vio_batch_set_tune(self.handle, ctypes.byref(t)), "set_tune")

    def get_tune(self) -> tuple[int, int, int, int, int, int]:
        """(k2_threads, pyr_tile_shift, stereo_after_select, pyr_first_levels, k1_threads,
        det_warps)."""
        t = BatchTune()
        _check(load().vio_batch_get_tune(self.handle, ctypes.byref(t)), "get_tune")
        return (t.k2_threads, t.pyr_tile_shift, t.stereo_after_select, t.pyr_first_levels,
                t.k1_threads, t.det_warps)

    def autotune(self, reps: int = 3, stream=None) -> float:
        ms = ctypes.c_float()
        _check(load().vio_batch_autotune(self.handle, reps, _stream(stream), ctypes.byref(ms)),
               "vio_batch_autotune")
        return float(ms.value)

    def reset_stream(self, g: int, s: int, stream=None):
        _check(load().vio_batch_reset_stream(self.handle, g, s, _stream(stream)), "reset")

    def launches_per_step(self) -> int:
        return int(load().vio_batch_launches_per_step(self.handle))

    def read_stats(self, g: int):
        """(ring array (STATS_RING, n_streams_g, len(STAT_NAMES)), steps run)."""
        import numpy as np
        n = self.groups[g][2]
        out = np.zeros((STATS_RING, n, len(STAT_NAMES)), np.int32)
        steps = ctypes.c_int64()
        _check(load().vio_batch_read_stats(self.handle, g, out.ctypes.data_as(ctypes.c_void_p),
                                           ctypes.byref(steps)), "vio_batch_read_stats")
        return out, int(steps.value)

    def set_initnet(self, net: "InitNet | None"):
        """Learned start of temporal tracking for every stream (see Frontend)."""
        self._net = net
        _check(load().vio_batch_set_initnet(self.handle, _ptr(net.packed) if net else None,
                                            ctypes.byref(net.cfg) if net else None),
               "vio_batch_set_initnet")

    def view(self, g: int) -> dict:
        """Device tensors of group g's lists; 'parity' selects each stream's
        current lists: track_xy[parity[s], s, c]."""
        import numpy as np
        v = FrontendView()
        _, _, n, cap = self.groups[g]
        par = np.zeros(n, np.int32)
        _check(load().vio_batch_get_view(self.handle, g, ctypes.byref(v),
                                         par.ctypes.data_as(ctypes.c_void_p)), "get_view")
        dev = torch.device("cuda", torch.cuda.current_device())
        return {
            "track_xy": _alias(v.d_track_xy, (2, n, 2, cap, 2), torch.float32, dev),
            "track_id": _alias(v.d_track_id, (2, n, 2, cap), torch.int32, dev),
            "track_status": _alias(v.d_track_status, (2, n, 2, cap), torch.uint8, dev),
            "track_count": _alias(v.d_track_count, (2, n, 2), torch.int32, dev),
            "new_xy": _alias(v.d_new_xy, (n, cap, 2), torch.float32, dev),
            "new_count": _alias(v.d_new_count, (n,), torch.int32, dev),
            "parity": par,
        }

    def stream_lists(self, g: int, s: int):
        """(xy list per camera, id list per camera) of stream s of group g (host numpy)."""
        v = self.view(g)
        q = int(v["parity"][s])
        cnt = v["track_count"][q, s].cpu().numpy()
        xy = [v["track_xy"][q, s, c, : cnt[c]].cpu().numpy() for c in range(2)]
        ids = [v["track_id"][q, s, c, : cnt[c]].cpu().numpy() for c in range(2)]
        return xy, ids


# ------------------------------------------------------------------ serving --

SERVER_LAST = 1
DONE_FIELDS = ("session", "tag", "t_arrival", "t_launch", "t_done", "n_tracks0", "n_tracks1",
               "n_new", "status")


def _groups_array(classes):
    arr = (StreamGroup * len(classes))()
    for i, (p, w, h, n, cap) in enumerate(classes):
        arr[i].params = p
        arr[i].w, arr[i].h, arr[i].n_streams, arr[i].capacity = w, h, n, cap
    return arr


def _hptr(a):
    """Address of a contiguous host buffer (numpy array or CPU tensor)."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor")
        return ctypes.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a contiguous array")
    return ctypes.c_void_p(a.ctypes.data)


def batch_device_bytes(classes) -> int:
    b = ctypes.c_int64()
    _check(load().vio_batch_device_bytes(_groups_array(classes), len(classes), ctypes.byref(b)),
           "vio_batch_device_bytes")
    return int(b.value)


def server_plan(classes, budget_bytes: int):
    """(slots per class, device bytes) that vio_server_create would use; raises
    VioError (out of memory) if one slot per class exceeds the budget."""
    import numpy as np
    slots = np.zeros(len(classes), np.int32)
    b = ctypes.c_int64()
    _check(load().vio_server_plan(_groups_array(classes), len(classes), int(budget_bytes),
                                  slots.ctypes.data_as(ctypes.c_void_p), ctypes.byref(b)),
           "vio_server_plan")
    return slots.tolist(), int(b.value)


def server_now() -> float:
    return float(load().vio_server_now())


def _done_rows(arr, n):
    import numpy as np
    out = np.zeros(n, dtype=[(k, np.float64 if k.startswith("t_") else np.int64)
                             for k in DONE_FIELDS])
    for i in range(n):
        d = arr[i]
        out[i] = (d.session, d.tag, d.t_arrival, d.t_launch, d.t_done, d.n_tracks[0],
                  d.n_tracks[1], d.n_new, d.status)
    return out


class Server:
    """vio_server: sessions of a few size classes, admitted by a device-memory
    budget, served by continuous batching. classes: list of (params, w, h,
    sessions wanted, capacity). Host frames must be pinned."""

    def __init__(self, classes, budget_bytes: int):
        self.classes = [(w, h, n, cap) for (_, w, h, n, cap) in classes]
        hdl = ctypes.c_void_p()
        _check(load().vio_server_create(ctypes.byref(hdl), _groups_array(classes), len(classes),
                                        int(budget_bytes)), "vio_server_create")
        self.handle = hdl
        self._keep = {}

    def close_server(self):
        if self.handle:
            load().vio_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close_server()
        except Exception:
            pass

    def slots(self, cls: int):
        n = ctypes.c_int32()
        b = ctypes.c_int64()
        _check(load().vio_server_slots(self.handle, cls, ctypes.byref(n), ctypes.byref(b)),
               "vio_server_slots")
        return int(n.value), int(b.value)

    def set_initnet(self, net: "InitNet | None"):
        self._net = net
        _check(load().vio_server_set_initnet(self.handle, _ptr(net.packed) if net else None,
                                             ctypes.byref(net.cfg) if net else None),
               "vio_server_set_initnet")

    def set_tune(self, k2_threads: int, pyr_tile_shift: int, stereo_after_select: int = 0,
                 pyr_first_levels: int = 0, k1_threads: int = 256, det_warps: int = 4):
        t = BatchTune(k2_threads, pyr_tile_shift, stereo_after_select, pyr_first_levels,
                      k1_threads, det_warps)
        _check(load().vio_server_set_tune(self.handle, ctypes.byref(t)), "vio_server_set_tune")

    def open(self, cls: int):
        sid = ctypes.c_int64()
        adm = ctypes.c_int32()
        _check(load().vio_server_open(self.handle, cls, ctypes.byref(sid), ctypes.byref(adm)),
               "vio_server_open")
        return int(sid.value), bool(adm.value)

    def set_output(self, session: int, xy, ids, count):
        self._keep[("out", session)] = (xy, ids, count)
        _check(load().vio_server_set_output(self.handle, session, _hptr(xy), _hptr(ids),
                                            _hptr(count)), "vio_server_set_output")

    def submit(self, session: int, frame, t_arrival: float, tag: int, flags: int = 0):
        _check(load().vio_server_submit(self.handle, session, _hptr(frame), t_arrival, tag,
                                        flags), "vio_server_submit")

    def close(self, session: int):
        _check(load().vio_server_close(self.handle, session), "vio_server_close")

    def poll(self) -> int:
        n = ctypes.c_int32()
        _check(load().vio_server_poll(self.handle, ctypes.byref(n)), "vio_server_poll")
        return int(n.value)

    def take(self, max_n: int = 1024):
        arr = (ServerDone * max_n)()
        n = load().vio_server_take(self.handle, arr, max_n)
        return _done_rows(arr, n)

    def run_trace(self, reqs, timeout_s: float = 600.0):
        """reqs: list of (session, t_offset, pinned frame, tag, flags), ascending
        t_offset. Returns (completions structured array, steps run)."""
        n = len(reqs)
        arr = (ServerReq * max(n, 1))()
        for i, (sid, t, fr, tag, fl) in enumerate(reqs):
            arr[i].session, arr[i].t_offset = sid, t
            arr[i].host_frame = _hptr(fr).value
            arr[i].tag, arr[i].flags = tag, fl
        out = (ServerDone * max(n, 1))()
        steps = ctypes.c_int64()
        _check(load().vio_server_run_trace(self.handle, arr, n, out, timeout_s,
                                           ctypes.byref(steps)), "vio_server_run_trace")
        return _done_rows(out, n), int(steps.value)

    def set_loop_policy(self, pin_cpu=-1, rt_priority=0):
        """vio_server_set_loop_policy: pin the trace loop's thread to a CPU
        (-2: the one it starts on) and run it at a SCHED_FIFO priority, where
        permitted."""
        _check(load().vio_server_set_loop_policy(self.handle, pin_cpu, rt_priority),
               "vio_server_set_loop_policy")

    def loop_policy_granted(self):
        """(pinned, real_time) as the last trace got them."""
        g = ctypes.c_int32()
        _check(load().vio_server_loop_policy_granted(self.handle, ctypes.byref(g)),
               "vio_server_loop_policy_granted")
        return bool(g.value & 1), bool(g.value & 2)

    def loop_stats(self):
        """(longest gap between passes of the last trace's host loop in seconds,
        passes longer than 1 ms)."""
        gap, n = ctypes.c_double(), ctypes.c_int64()
        _check(load().vio_server_loop_stats(self.handle, ctypes.byref(gap), ctypes.byref(n)),
               "vio_server_loop_stats")
        return float(gap.value), int(n.value)
