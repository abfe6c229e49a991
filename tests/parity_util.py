"""Shared helpers of the GPU parity tests: comparison rules for track results.

Flow tolerance: 1e-3 px against the FP64 oracle. A status disagreement is
accepted only when the oracle shows the decision sat on its threshold: the
forward-backward distance within 1e-3 px of the threshold, or a bounds test
within 1e-3 px (level-0) of its bound."""
from __future__ import annotations

import numpy as np

FLOW_TOL = 1e-3
BAND = 1e-3


def compare_tracks(g_xy, g_status, ref, fb_max_dist, min_agree=0.999):
    """g_xy (n,2) GPU forward positions, g_status (n,), ref: oracle.track dict.
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
    return {"n": n, "agree": float(agree.mean()) if n else 1.0,
            "n_disagree": int((~agree).sum()), "max_err": float(err),
            "n_ok": int((o_status == 0).sum())}
