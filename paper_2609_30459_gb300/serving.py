"""Host-side helpers of the serving loop (vio_server): Poisson request traces
and latency summaries. The loop itself is native (csrc/server.cu); these
functions only prepare its input and read its output.
"""
from __future__ import annotations

import numpy as np


def pingpong(n_frames: int, k: int) -> int:
    """Index of the k-th frame when a pool of n_frames is played forward and
    back (motion stays continuous when the pool wraps)."""
    if n_frames <= 1:
        return 0
    period = 2 * n_frames - 2
    r = k % period
    return r if r < n_frames else period - r


def poisson_trace(rates_hz, duration_s: float, seed: int, max_frames=None):
    """Arrival times of frame requests: session i sends frames as a Poisson
    process of rate rates_hz[i] over [0, duration_s) (exponential gaps), at
    most max_frames[i] of them if given. Returns a list of (t, session, k)
    with k the session's frame number, in ascending t (ties by session)."""
    rng = np.random.default_rng(seed)
    out = []
    for i, lam in enumerate(rates_hz):
        t, k = 0.0, 0
        cap = None if max_frames is None else max_frames[i]
        while True:
            t += rng.exponential(1.0 / lam)
            if t >= duration_s or (cap is not None and k >= cap):
                break
            out.append((t, i, k))
            k += 1
    out.sort(key=lambda r: (r[0], r[1]))
    return out


def latency_summary(done) -> dict:
    """p50/p99/max latency (arrival -> completion), queueing (arrival ->
    launch) and aggregate frames/s of a structured completion array."""
    if len(done) == 0:
        return {"frames": 0}
    lat = done["t_done"] - done["t_arrival"]
    queue = done["t_launch"] - done["t_arrival"]
    span = done["t_done"].max() - done["t_arrival"].min()
    return {"frames": int(len(done)),
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "max_ms": float(lat.max() * 1e3),
            "queue_p50_ms": float(np.percentile(queue, 50) * 1e3),
            "queue_p99_ms": float(np.percentile(queue, 99) * 1e3),
            "frames_per_s": float(len(done) / span) if span > 0 else None,
            "failed": int((done["status"] != 0).sum())}
