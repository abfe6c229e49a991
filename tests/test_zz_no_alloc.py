"""vio_detect_grid_noalloc, the detection entry point for callers that cannot
allocate device memory (for example code running inside a fixed memory pool or
a host runtime that owns every allocation): called three times in a row (twice
through the C ABI, then through the Python binding with a per-pixel mask on
several images), each result must equal vio_detect_grid's on the same inputs
(detection is integer work, so the comparison is exact). The scratch array is
shared by all calls and keeps the previous call's contents, which the later
calls exercise. Oversized calls are rejected whether the slots come from the
image count, k or the cell size. This file is collected last on purpose."""
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


def _run_both(params, imgs, occ, cap, mask=None, wrapper=False):
    n = imgs.shape[0]
    h, w = imgs.shape[1], imgs.shape[2]
    pyr = vio.Pyramids(imgs, 1)
    ref_kp = torch.full((n, cap, 2), -7.0, device="cuda")
    ref_sc = torch.full((n, cap), -7, dtype=torch.int16, device="cuda")
    ref_n = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    ctx = vio.Context(params, w, h, n)
    ctx.detect_grid(pyr, pyr.batch(), ref_kp, ref_sc, ref_n, cap, occupancy=occ, mask=mask,
                    mask_stride=w * h)
    kp = torch.full((n, cap, 2), -9.0, device="cuda")
    sc = torch.full((n, cap), -9, dtype=torch.int16, device="cuda")
    cnt = torch.full((n,), -9, dtype=torch.int32, device="cuda")
    if wrapper:       # the Python binding of the same entry point
        vio.detect_grid_noalloc(params, pyr, pyr.batch(), kp, sc, cnt, cap, occupancy=occ,
                                mask=mask, mask_stride=w * h)
    else:
        st = vio.load().vio_detect_grid_noalloc(
            ctypes.byref(params), ctypes.byref(pyr.layout), ctypes.byref(pyr.batch()),
            ctypes.c_void_p(occ.data_ptr()) if occ is not None else None,
            ctypes.c_void_p(mask.data_ptr()) if mask is not None else None, w * h,
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
    # call 3, through the Python binding: a seeded per-pixel mask on three
    # images (the mask's image stride is exercised), k = 3
    p3 = vio.default_params(n_levels=1, cell_w=50, cell_h=40, k_per_cell=3)
    h, w = 240, 320
    mask = torch.from_numpy((np.random.default_rng(9).random((3, h, w)) > 0.3)
                            .astype(np.uint8)).cuda()
    _run_both(p3, _images(31, 3, h, w), None, (w // 50) * (h // 40) * 3, mask=mask,
              wrapper=True)


def _noalloc_status(p, imgs):
    pyr = vio.Pyramids(imgs, 1)
    out = torch.zeros(16, device="cuda")
    st = vio.load().vio_detect_grid_noalloc(
        ctypes.byref(p), ctypes.byref(pyr.layout), ctypes.byref(pyr.batch()), None, None, 0,
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), 1, None)
    torch.cuda.synchronize()
    return st


def test_noalloc_rejects_oversized_calls():
    limit = 65536                               # VIO_NOALLOC_MAX_CELL_SLOTS
    # through the image count: 2 images x 4096 cells x k 8 = 65536 slots fits,
    # a third image does not
    p = vio.default_params(n_levels=1, cell_w=4, cell_h=4, k_per_cell=8)
    assert _noalloc_status(p, torch.zeros((2, 256, 256), dtype=torch.uint8,
                                          device="cuda")) == vio.OK
    assert _noalloc_status(p, torch.zeros((3, 256, 256), dtype=torch.uint8,
                                          device="cuda")) == vio.ERR_UNSUPPORTED
    # through k: 8193 cells x k 8 = 65544 slots, while k 7 (57351) fits
    img = torch.zeros((1, 1, 8193), dtype=torch.uint8, device="cuda")
    p8 = vio.default_params(n_levels=1, cell_w=1, cell_h=1, k_per_cell=8, detect_border=0)
    assert 8193 * 8 > limit
    assert _noalloc_status(p8, img) == vio.ERR_UNSUPPORTED
    p7 = vio.default_params(n_levels=1, cell_w=1, cell_h=1, k_per_cell=7, detect_border=0)
    assert _noalloc_status(p7, img) == vio.OK
    # through the cell size: exactly limit + 1 cells of 1 x 1 px with k = 1 are
    # rejected, limit cells fit
    p1 = vio.default_params(n_levels=1, cell_w=1, cell_h=1, k_per_cell=1, detect_border=0)
    assert _noalloc_status(p1, torch.zeros((1, 1, limit + 1), dtype=torch.uint8,
                                           device="cuda")) == vio.ERR_UNSUPPORTED
    assert _noalloc_status(p1, torch.zeros((1, 1, limit), dtype=torch.uint8,
                                           device="cuda")) == vio.OK
