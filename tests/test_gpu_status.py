"""The device status word and the bounded device-side wait (vio_wait_flag,
vio_ctx_sync, vio_last_error): a wait on a flag that nothing sets gives up
after its limit, records VIO_ERR_TIMEOUT in the status word and ends, and the
context stays usable afterwards (a detection on it still matches the oracle).
No GPU fault is involved: the kernel itself stops waiting."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2609_30459_gb300 import synth

pytestmark = pytest.mark.gpu

vio = pytest.importorskip("paper_2609_30459_gb300.vio")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vio.load(build=True)
    oracle.build()


def test_wait_on_an_unset_flag_times_out_and_the_context_survives():
    w, h = 320, 240
    p = vio.default_params(n_levels=1, cell_w=40, cell_h=40)
    ctx = vio.Context(p, w, h, 1)
    assert ctx.last_error() == vio.OK
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    ctx.wait_flag(flag, 1, 50_000_000)                 # 50 ms, nothing sets the flag
    e1.record(s)
    assert ctx.sync() == vio.ERR_TIMEOUT
    waited = e0.elapsed_time(e1)
    assert 45.0 <= waited < 2000.0, waited
    # read and cleared by the sync
    assert ctx.last_error() == vio.OK
    # a flag that is set ends the wait at once, with no error
    flag.fill_(1)
    t0 = time.perf_counter()
    ctx.wait_flag(flag, 1, 1_500_000_000)
    assert ctx.sync() == vio.OK
    assert time.perf_counter() - t0 < 1.0
    # the context still works
    img = synth.quantize(synth.band_limited_texture(3, h, w), np.random.default_rng(0), 2.0)
    pyr = vio.Pyramids(torch.from_numpy(img[None]).cuda(), 1)
    cap = (w // 40) * (h // 40)
    kp = torch.zeros((1, cap, 2), device="cuda")
    sc = torch.zeros((1, cap), dtype=torch.int16, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.detect_grid(pyr, pyr.batch(), kp, sc, cnt, cap)
    assert ctx.sync() == vio.OK
    rk, _ = oracle.detect_grid(img, 40, 40, border=p.detect_border)
    assert int(cnt[0]) == len(rk) and np.array_equal(kp[0, :len(rk)].cpu().numpy(), rk)
    ctx.close()


def test_wait_rejects_bad_arguments():
    p = vio.default_params(n_levels=1, cell_w=40, cell_h=40)
    ctx = vio.Context(p, 64, 64, 1)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(vio.VioError):
        ctx.wait_flag(flag, 1, -1)
    with pytest.raises(vio.VioError):
        ctx.wait_flag(flag, 1, 3_000_000_000)
    ctx.close()
