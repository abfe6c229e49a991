"""Host logic of the serving loop, without a GPU: the memory plan of
vio_server (a host-only call of the library) and the Poisson traces."""
import numpy as np
import pytest

from paper_2609_30459_gb300 import serving


def _lib():
    from paper_2609_30459_gb300 import build_lib, vio
    build_lib.build()
    vio.load()
    return vio


def _classes(vio, n=8):
    return [(vio.default_params(n_levels=5, cell_w=32, cell_h=32), 640, 480, n, 600),
            (vio.default_params(n_levels=5, cell_w=48, cell_h=43), 1920, 1080, n, 2000)]


def test_plan_fits_the_budget():
    vio = _lib()
    cl = _classes(vio)
    full_slots, full = vio.server_plan(cl, 1 << 40)
    assert full_slots == [8, 8]
    # per-slot bytes: the batch's own size for one stream plus two staging frames
    one = [vio.batch_device_bytes([c[:3] + (1,) + c[4:]]) for c in cl]
    assert full >= sum(8 * (b + 2 * 2 * c[1] * c[2]) for b, c in zip(one, cl))
    for frac in (0.9, 0.5, 0.26):
        slots, used = vio.server_plan(cl, int(full * frac))
        assert used <= int(full * frac)
        assert all(1 <= s <= 8 for s in slots) and slots != [8, 8]
    with pytest.raises(vio.VioError):
        vio.server_plan(cl, 1 << 20)                 # not even one slot per class


def test_plan_rejects_invalid_classes():
    vio = _lib()
    bad = [(vio.default_params(n_levels=5, cell_w=32, cell_h=32), 640, 480, 0, 600)]
    with pytest.raises(vio.VioError):
        vio.server_plan(bad, 1 << 30)


def test_poisson_trace_rates_and_order():
    rates = [30.0, 200.0, 80.0]
    tr = serving.poisson_trace(rates, 50.0, seed=3)
    t = np.array([r[0] for r in tr])
    assert np.all(np.diff(t) >= 0) and t.min() >= 0 and t.max() < 50.0
    for i, lam in enumerate(rates):
        ks = [r[2] for r in tr if r[1] == i]
        assert ks == list(range(len(ks)))            # frames in order, none skipped
        # Poisson count over 50 s: mean 50*lam, sd sqrt(50*lam)
        assert abs(len(ks) - 50 * lam) < 5 * np.sqrt(50 * lam)
    capped = serving.poisson_trace(rates, 50.0, seed=3, max_frames=[5, 5, 5])
    assert all(sum(1 for r in capped if r[1] == i) == 5 for i in range(3))


def test_pingpong_and_summary():
    assert [serving.pingpong(4, k) for k in range(8)] == [0, 1, 2, 3, 2, 1, 0, 1]
    assert serving.pingpong(1, 5) == 0
    dt = [(k, np.float64 if k.startswith("t_") else np.int64) for k in
          ("session", "tag", "t_arrival", "t_launch", "t_done", "n_tracks0", "n_tracks1",
           "n_new", "status")]
    d = np.zeros(100, dtype=dt)
    d["t_arrival"] = np.arange(100) * 0.01
    d["t_launch"] = d["t_arrival"] + 0.001
    d["t_done"] = d["t_arrival"] + 0.002
    d["t_done"][-1] += 0.1
    s = serving.latency_summary(d)
    assert s["p50_ms"] == pytest.approx(2.0) and s["max_ms"] == pytest.approx(102.0)
    assert s["queue_p50_ms"] == pytest.approx(1.0) and s["failed"] == 0
