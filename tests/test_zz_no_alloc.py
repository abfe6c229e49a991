"""vio_detect_grid_noalloc, the detection entry point for callers that cannot
allocate device memory (for example code running inside a fixed memory pool or
a host runtime that owns every allocation): called through the C ABI twice in
a row, each result must equal vio_detect_grid's on the same inputs (detection
is integer work, so the comparison is exact). The scratch array is shared by
all calls and keeps the previous call's contents, which the second call
exercises. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2609_30459_gb300 import synth

pytestmark = pytest.mark.gpu

vio = pytest.importorskip("paper_2609_30459_gb300.vio")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vio.load(build=True)


def _images(seed, n, h, w):
    rng = np.random.default_rng(seed)
    imgs = np.stack([synth.quantize(synth.band_limited_texture(seed + i, h, w, 1.5), rng, 2.0)
                     for i in range(n)])
    return torch.from_numpy(imgs).cuda()


def _run_both(params, imgs, occ, cap):
    n = imgs.shape[0]
    pyr = vio.Pyramids(imgs, 1)
    ref_kp = torch.full((n, cap, 2), -7.0, device="cuda")
    ref_sc = torch.full((n, cap), -7, dtype=torch.int16, device="cuda")
    ref_n = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    ctx = vio.Context(params, imgs.shape[2], imgs.shape[1], n)
    ctx.detect_grid(pyr, pyr.batch(), ref_kp, ref_sc, ref_n, cap, occupancy=occ)
    kp = torch.full((n, cap, 2), -9.0, device="cuda")
    sc = torch.full((n, cap), -9, dtype=torch.int16, device="cuda")
    cnt = torch.full((n,), -9, dtype=torch.int32, device="cuda")
    st = vio.load().vio_detect_grid_noalloc(
        ctypes.byref(params), ctypes.byref(pyr.layout), ctypes.byref(pyr.batch()),
        ctypes.c_void_p(occ.data_ptr()) if occ is not None else None, None, 0,
        ctypes.c_void_p(kp.data_ptr()), ctypes.c_void_p(sc.data_ptr()),
        ctypes.c_void_p(cnt.data_ptr()), cap,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == vio.OK
    torch.cuda.synchronize()
    ctx.close()
    assert torch.equal(cnt, ref_n)
    for i in range(n):
        c = int(ref_n[i])
        assert c > 0
        assert torch.equal(kp[i, :c], ref_kp[i, :c])
        assert torch.equal(sc[i, :c], ref_sc[i, :c])


def test_noalloc_matches_detect_grid_two_calls_in_a_row():
    # call 1: k = 2 on three 752x480 images, no occupancy
    p1 = vio.default_params(n_levels=1, cell_w=94, cell_h=60, k_per_cell=2)
    _run_both(p1, _images(11, 3, 480, 752), None, 8 * 8 * 2)
    # call 2: different size, cells, k and occupancy; the shared scratch still
    # holds call 1's candidates
    p2 = vio.default_params(n_levels=1, cell_w=37, cell_h=32, k_per_cell=1)
    h, w = 360, 600
    gx, gy = w // 37, h // 32
    occ = torch.from_numpy(np.random.default_rng(5).integers(0, 2, (2, gx * gy))
                           .astype(np.uint8)).cuda()
    _run_both(p2, _images(23, 2, h, w), occ, gx * gy)


def test_noalloc_rejects_oversized_calls():
    p = vio.default_params(n_levels=1, cell_w=4, cell_h=4, k_per_cell=8)
    imgs = torch.zeros((2, 256, 256), dtype=torch.uint8, device="cuda")
    pyr = vio.Pyramids(imgs, 1)
    out = torch.zeros(16, device="cuda")
    st = vio.load().vio_detect_grid_noalloc(
        ctypes.byref(p), ctypes.byref(pyr.layout), ctypes.byref(pyr.batch()), None, None, 0,
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), 1, None)
    # 2 images x 4096 cells x k 8 = 65536 slots fits; 2 x 4096 x 8 + more does not
    assert st == vio.OK
    torch.cuda.synchronize()
    imgs3 = torch.zeros((3, 256, 256), dtype=torch.uint8, device="cuda")
    pyr3 = vio.Pyramids(imgs3, 1)
    st = vio.load().vio_detect_grid_noalloc(
        ctypes.byref(p), ctypes.byref(pyr3.layout), ctypes.byref(pyr3.batch()), None, None, 0,
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), 1, None)
    assert st == vio.ERR_UNSUPPORTED
