"""Shared helpers of the GPU parity tests: comparison rules for track results.

Flow tolerance: 1e-3 px against the FP64 oracle. A status disagreement is
accepted only when the oracle shows the decision sat on its threshold: the
forward-backward distance within 1e-3 px of the threshold, or a bounds test
within 1e-3 px (level-0) of its bound.

Rotation tolerance: turning the 52-point pattern by d_theta moves its
outermost point (radius sqrt(7^2 + 3^2) = 7.62 px at level 0) by 7.62 d_theta
px, so the angle is held to the rotation that moves that point by FLOW_TOL."""
from __future__ import annotations

import numpy as np

FLOW_TOL = 1e-3
BAND = 1e-3
THETA_TOL = FLOW_TOL / np.hypot(7.0, 3.0)


def compare_tracks(g_xy, g_status, ref, fb_max_dist, min_agree=0.999, g_theta=None):
    """g_xy (n,2) GPU forward positions, g_status (n,), ref: oracle.track dict,
    g_theta (n,) GPU forward angles or None (calls that return no angle).
    Returns a dict of statistics; raises AssertionError on a parity failure."""
    g_xy = np.asarray(g_xy, np.float64)
    g_status = np.asarray(g_status)
    o_status = ref["status"]
    n = len(o_status)
    agree = g_status == o_status
    explained = np.zeros(n, bool)
    fbd = ref["fb_dist"]
    with np.errstate(invalid="ignore"):
        explained |= np.abs(fbd - fb_max_dist) <= BAND
    explained |= ref["margin"] <= BAND
    bad = ~agree & ~explained
    assert not bad.any(), (
        f"{bad.sum()} unexplained status disagreements: gpu {g_status[bad][:10]} "
        f"oracle {o_status[bad][:10]} margin {ref['margin'][bad][:10]} "
        f"fb {fbd[bad][:10]}")
    if n >= 1000:
        assert agree.mean() >= min_agree, agree.mean()
    # flow: wherever both have a forward result (OK or FB_FAIL on both sides)
    have = agree & np.isin(o_status, (0, 5))
    err = np.abs(g_xy[have] - ref["warp"][have, :2]).max() if have.any() else 0.0
    assert err < FLOW_TOL, f"flow differs by {err} px"
    th_err = 0.0
    if g_theta is not None and have.any():
        th_err = float(np.abs(np.asarray(g_theta, np.float64)[have] - ref["warp"][have, 2]).max())
        assert th_err < THETA_TOL, f"angle differs by {th_err} rad"
    return {"n": n, "agree": float(agree.mean()) if n else 1.0,
            "n_disagree": int((~agree).sum()), "max_err": float(err),
            "max_theta_err": th_err, "n_ok": int((o_status == 0).sum())}
