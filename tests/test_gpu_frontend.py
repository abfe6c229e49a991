"""GPU parity of the per-frame frontend (Sec. III-B) against the oracle's
frontend, step by step: before each frame the oracle is given the GPU's state
(keypoint lists and ids), so that one step's outputs are compared on the same
inputs and a status decision on a threshold does not carry over."""
import numpy as np
import pytest
import torch

import oracle
from oracle import frontend as ofe
from paper_2609_30459_gb300 import synth
from tests.parity_util import BAND, FLOW_TOL

pytestmark = pytest.mark.gpu

vio = pytest.importorskip("paper_2609_30459_gb300.vio")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vio.load(build=True)
    oracle.build()


def _check_track_lists(g_xy, g_id, o_xy, o_id, explained_ids):
    """Same ids in the same order, except ids whose decision was on a
    threshold; positions of common ids within FLOW_TOL."""
    gs, os_ = list(g_id), list(o_id)
    diff = set(gs) ^ set(os_)
    assert diff <= explained_ids, (sorted(diff - explained_ids)[:10], len(diff))
    gpos = {i: p for i, p in zip(gs, g_xy)}
    opos = {i: p for i, p in zip(os_, o_xy)}
    common = [i for i in gs if i in opos]
    assert [i for i in gs if i in opos] == [i for i in os_ if i in gpos]   # same order
    if common:
        err = max(np.abs(np.asarray(gpos[i], np.float64) - opos[i]).max() for i in common)
        assert err < FLOW_TOL, err
        return err
    return 0.0


def _explained(res, ids, fb_max):
    if res is None:
        return set()
    with np.errstate(invalid="ignore"):
        m = (np.abs(res["fb_dist"] - fb_max) <= BAND) | (res["margin"] <= BAND)
    return set(np.asarray(ids)[m].tolist())


# Step-by-step cases: (w, h, levels, cell w, cell h, k, frames, max motion px,
# stereo streams, thresholds, Gauss-Newton iterations).
#  cfg2_small: the 752x480 sequence workload (4 levels, 20x15 cells, k = 1);
#  cfg1_k2:    cfg 1 (3 levels, 8x8 cells of 94x60, k = 2, small motion);
#  cfg3_rig:   the high-pixel rig, two stereo pairs at 1920x1080, 5 levels,
#              40x25 cells of 48x43 px (1000 keypoints per image), motion 40 px;
#  lite:       the paper's lite parameters (Sec. IV-D): minimum FAST threshold
#              20, 82-px cells, 3 Gauss-Newton iterations.
FRONTEND_CASES = {
    "cfg2_small": (752, 480, 4, 37, 32, 1, 8, 15.0, 1, (40, 20, 10, 5), 5),
    "cfg1_k2": (752, 480, 3, 94, 60, 2, 4, 3.0, 1, (40, 20, 10, 5), 5),
    "cfg3_rig": (1920, 1080, 5, 48, 43, 1, 3, 40.0, 2, (40, 20, 10, 5), 5),
    "lite": (752, 480, 4, 82, 82, 1, 8, 15.0, 1, (40, 20), 3),
}


@pytest.mark.parametrize("cfg", list(FRONTEND_CASES))
def test_frontend_steps_match_oracle(cfg):
    w, h, L, cw, ch, k, n_frames, motion, ns, thr, gn = FRONTEND_CASES[cfg]
    seq = synth.make_sequence(4000 + n_frames, n_frames, w, h, ns, max_motion=motion,
                              tex_size=2048)
    p = vio.default_params(n_levels=L, cell_w=cw, cell_h=ch, k_per_cell=k, thresholds=thr,
                           gn_iters=gn)
    op = ofe.Params(n_levels=L, cell_w=cw, cell_h=ch, k=k, thresholds=thr, gn_iters=gn)
    cap = 2 * (w // cw) * (h // ch) * k
    fe = vio.Frontend(p, w, h, ns, cap)
    frames = torch.from_numpy(seq.frames).cuda().view(n_frames, ns, 2, h, w)
    states = [ofe.StreamState() for _ in range(ns)]
    prev_ids = [[np.zeros(0, np.int32), np.zeros(0, np.int32)] for _ in range(ns)]
    total_tracks = 0
    total_new = 0
    for t in range(n_frames):
        fe.step(frames[t])
        torch.cuda.synchronize()
        v = fe.view()
        for s in range(ns):
            st = states[s]
            img = seq.frames[t, 2 * s: 2 * s + 2]
            res = ofe.step(st, img, op, cap, n_threads=8)
            g_new = int(v["new_count"][s])
            g_new_xy = v["new_xy"][s, :g_new].cpu().numpy()
            cnt = v["track_count"][s].cpu().numpy()
            gx = [v["track_xy"][s, c, : cnt[c]].cpu().numpy() for c in range(2)]
            gi = [v["track_id"][s, c, : cnt[c]].cpu().numpy() for c in range(2)]
            # the GPU's camera-0 survivors come first in its list: their
            # occupancy, given to the oracle's detection, must give the GPU's
            # detections bit for bit (whatever the threshold decisions upstream)
            assert cnt[0] < cap            # no truncation: the survivors are cnt - new
            surv0 = int(cnt[0]) - g_new
            assert surv0 >= 0
            g_occ = ofe.occupancy(gx[0][:surv0], w, h, cw, ch)
            o_new_xy, _ = oracle.detect_grid(img[0], cw, ch, k=k, thresholds=thr,
                                             border=p.detect_border, occupancy=g_occ)
            assert np.array_equal(g_new_xy, o_new_xy), (t, s)
            assert np.array_equal(gx[0][surv0:], g_new_xy)
            total_new += g_new
            # temporal tracks and matches: explained differences only
            expl = set()
            for c in range(2):
                if res["track"][c] is not None:
                    expl |= _explained(res["track"][c], prev_ids[s][c], p.fb_max_dist)
            expl |= _explained(res["match"], st.ids[0][-len(res["new_xy"]):]
                               if len(res["new_xy"]) else [], p.fb_max_dist)
            for c in range(2):
                _check_track_lists(gx[c], gi[c], st.xy[c], st.ids[c], expl)
            total_tracks += int(cnt.sum())
            # hand the GPU state to the oracle for the next step
            st.xy = [gx[0].copy(), gx[1].copy()]
            st.ids = [gi[0].copy(), gi[1].copy()]
            prev_ids[s] = [gi[0].copy(), gi[1].copy()]
    assert total_tracks > 0 and total_new > 0
    fe.close()


def test_frontend_reset_and_two_streams():
    w, h, L = 320, 240, 3
    seq = synth.make_sequence(5001, 3, w, h, 2, max_motion=4.0, tex_size=1024)
    p = vio.default_params(n_levels=L, cell_w=40, cell_h=40)
    cap = 2 * (w // 40) * (h // 40)
    fe = vio.Frontend(p, w, h, 2, cap)
    frames = torch.from_numpy(seq.frames).cuda()                  # (F, 4, h, w): 2 streams
    for t in range(3):
        fe.step(frames[t].view(2, 2, h, w))
    torch.cuda.synchronize()
    c1 = fe.view()["track_count"].cpu().numpy().copy()
    # stream-independence: the same frames alone give the same lists
    fe_a = vio.Frontend(p, w, h, 1, cap)
    alone = [frames[t, 2:4].reshape(1, 2, h, w).contiguous() for t in range(3)]  # kept alive
    for t in range(3):
        fe_a.step(alone[t])
    torch.cuda.synchronize()
    va, vb = fe_a.view(), fe.view()
    assert np.array_equal(va["track_count"][0].cpu().numpy(), c1[1])
    for c in range(2):
        n = c1[1, c]
        assert torch.equal(va["track_xy"][0, c, :n], vb["track_xy"][1, c, :n])
        assert torch.equal(va["track_id"][0, c, :n], vb["track_id"][1, c, :n])
    fe.reset()
    torch.cuda.synchronize()
    assert (fe.view()["track_count"] == 0).all()


@pytest.mark.parametrize("learned", [False, True])
def test_frontend_pipelined_run_equals_steps(learned):
    """vio_frontend_run without stage timing overlaps the front of each step
    (pyramids, detection) with the tracking of the step before: same lists,
    ids and stats as one step at a time, also across several run calls."""
    w, h, L = 376, 240, 4
    n = 11
    seq = synth.make_sequence(5007, n, w, h, 1, max_motion=6.0, tex_size=1024)
    p = vio.default_params(n_levels=L, cell_w=47, cell_h=40)
    cap = 2 * (w // 47) * (h // 40)
    frames = torch.from_numpy(seq.frames).cuda().view(n, 1, 2, h, w)
    a, b = vio.Frontend(p, w, h, 1, cap), vio.Frontend(p, w, h, 1, cap)
    if learned:
        from paper_2609_30459_gb300 import initnet_train
        net = vio.InitNet.load(initnet_train.DEFAULT_WEIGHTS)
        a.set_initnet(net)
        b.set_initnet(net)
    for t in range(n):
        a.step(frames[t])
    b.run(frames[:4].contiguous())
    b.run(frames[4:].contiguous())
    torch.cuda.synchronize()
    va, vb = a.view(), b.view()
    assert torch.equal(va["track_count"], vb["track_count"])
    for c in range(2):
        nc = int(va["track_count"][0, c])
        assert nc > 0
        assert torch.equal(va["track_xy"][0, c, :nc], vb["track_xy"][0, c, :nc])
        assert torch.equal(va["track_id"][0, c, :nc], vb["track_id"][0, c, :nc])
    assert torch.equal(va["new_count"], vb["new_count"])
    sa, na = a.read_stats()
    sb, nb = b.read_stats()
    assert na == nb == n and np.array_equal(sa[:n], sb[:n])


def test_frontend_step_host_async_equals_step_host():
    """Pipelined host steps (uploads, fronts and the rest on the frontend's own
    streams, a done event per step) give each step's host outputs exactly as
    the plain host step, with a reset and a plain host step in between."""
    w, h, L = 376, 240, 4
    n, R = 10, 3
    seq = synth.make_sequence(5011, n, w, h, 1, max_motion=6.0, tex_size=1024)
    p = vio.default_params(n_levels=L, cell_w=47, cell_h=40)
    cap = 2 * (w // 47) * (h // 40)
    host = torch.from_numpy(seq.frames).view(n, 1, 2, h, w).pin_memory()
    a, b = vio.Frontend(p, w, h, 1, cap), vio.Frontend(p, w, h, 1, cap)
    da = torch.empty((R, 1, 2, h, w), dtype=torch.uint8, device="cuda")
    db = torch.empty_like(da)
    oa = [a.host_outputs() for _ in range(n)]
    ob = [b.host_outputs() for _ in range(n)]
    evs = [torch.cuda.Event() for _ in range(n)]
    for e in evs:
        e.record()
    for t in range(n):
        if t == 5:
            a.reset()
            b.reset()
        a.step_host(host[t], da[t % R], oa[t])
        if t == 7:
            b.step_host(host[t], db[t % R], ob[t])
        else:
            b.step_host_async(host[t], db[t % R], ob[t], evs[t])
    torch.cuda.synchronize()
    for t in range(n):
        assert torch.equal(oa[t]["count"], ob[t]["count"]), t
        assert torch.equal(oa[t]["new_count"], ob[t]["new_count"]), t
        for c in range(2):
            nc = int(oa[t]["count"][0, c])
            assert torch.equal(oa[t]["xy"][0, c, :nc], ob[t]["xy"][0, c, :nc]), (t, c)
            assert torch.equal(oa[t]["id"][0, c, :nc], ob[t]["id"][0, c, :nc]), (t, c)
        nn = int(oa[t]["new_count"][0])
        assert torch.equal(oa[t]["new_xy"][0, :nn], ob[t]["new_xy"][0, :nn]), t
    assert int(oa[n - 1]["count"].sum()) > 0


def test_frontend_run_equals_steps():
    w, h, L = 376, 240, 3
    seq = synth.make_sequence(5003, 6, w, h, 1, max_motion=5.0, tex_size=1024)
    p = vio.default_params(n_levels=L, cell_w=47, cell_h=40)
    cap = 2 * (w // 47) * (h // 40)
    frames = torch.from_numpy(seq.frames).cuda().view(6, 1, 2, h, w)
    a, b = vio.Frontend(p, w, h, 1, cap), vio.Frontend(p, w, h, 1, cap)
    for t in range(6):
        a.step(frames[t])
    b.set_timing(True)
    b.run(frames)
    torch.cuda.synchronize()
    stage_ms, n, per_step = b.read_timing(max_steps=6)
    assert n == 6 and len(per_step) == 6 and all(x > 0 for x in per_step)
    va, vb = a.view(), b.view()
    assert torch.equal(va["track_count"], vb["track_count"])
    n0, n1 = va["track_count"][0].tolist()
    for c, nc in ((0, n0), (1, n1)):
        assert torch.equal(va["track_xy"][0, c, :nc], vb["track_xy"][0, c, :nc])
        assert torch.equal(va["track_id"][0, c, :nc], vb["track_id"][0, c, :nc])
    stats, steps = b.read_stats()
    assert steps == 6 and stats[5, 0, 4] == int(vb["new_count"][0])
    # step-only timing: the same lists, per-step times, no stage times
    c = vio.Frontend(p, w, h, 1, cap)
    c.set_timing(2)
    c.run(frames)
    torch.cuda.synchronize()
    stage_ms, n, per_step = c.read_timing(max_steps=6)
    assert n == 6 and all(x > 0 for x in per_step) and all(v == 0 for v in stage_ms.values())
    vc = c.view()
    assert torch.equal(va["track_count"], vc["track_count"])
    for cam, nc in ((0, n0), (1, n1)):
        assert torch.equal(va["track_xy"][0, cam, :nc], vc["track_xy"][0, cam, :nc])
    c.close()


# ------------------------------------------------ learned start of tracking ---

CONF_BAND = 1e-3   # |GPU - oracle| confidence: <= 0.25 * the raw-output tolerance


def _band(res, fb_max):
    with np.errstate(invalid="ignore"):
        return (np.abs(res["fb_dist"] - fb_max) <= BAND) | (res["margin"] <= BAND)


def _explained_net(res, ids, fb_max, tau):
    """Ids whose outcome may differ: confidence on the gate, or a threshold
    decision of the proposed or the plain track."""
    if res is None:
        return set()
    ids = np.asarray(ids)
    m = np.abs(res["conf"] - tau) <= CONF_BAND
    gate, rl = res["learned_track"]
    if rl is not None:
        m[gate] |= _band(rl, fb_max)
    rest, rp = res["plain_track"]
    if rp is not None:
        m[rest] |= _band(rp, fb_max)
    return set(ids[m].tolist())


def _net_master(kind):
    from oracle import initnet as onet
    rng = np.random.default_rng(12)
    if kind == "const":
        # all weights zero: every proposal is zero flow with confidence 0.95
        p = {k: np.zeros(onet.SHAPES[k]) for k in onet.ORDER}
        p["b5"] = np.array([0.0, 0.0, 3.0])
    else:
        fan = {"w1": 36, "w2": 288, "w3": 288, "w4": 128, "w5": 64}
        p = {k: (rng.normal(0, np.sqrt(2.0 / fan[k]), onet.SHAPES[k]) if k in fan
                 else rng.normal(0, 0.1, onet.SHAPES[k])) for k in onet.ORDER}
        p["b5"] = np.array([0.0, 0.0, 0.0])
    flat = onet.flatten(p).astype(np.float32)
    q = onet.unflatten(flat.astype(np.float64))
    q = {k: (onet.bf16_round(v) if k.startswith("w") else v) for k, v in q.items()}
    return flat, q


@pytest.mark.parametrize("kind", ["const", "random"])
def test_frontend_learned_start_matches_oracle(kind):
    """Positions within 1e-3 px of the oracle's. A learned track counts only
    when it has converged (its last level-0 step below the gate), so it sits
    at the optimum its start leads to whatever the proposal's last bits; the
    only positions that may differ are those whose oracle result had not
    converged (last step above the gate: not determined to 1e-3 px), where the
    two sides may also have taken different paths (few, counted)."""
    w, h, L, cw, ch, n_frames, motion = 640, 480, 5, 32, 32, 5, 12.0
    seq = synth.make_sequence(4100, n_frames, w, h, 1, max_motion=motion, tex_size=2048)
    p = vio.default_params(n_levels=L, cell_w=cw, cell_h=ch)
    op = ofe.Params(n_levels=L, cell_w=cw, cell_h=ch)
    cap = 2 * (w // cw) * (h // ch)
    flat, q = _net_master(kind)
    tau = 0.5
    net = vio.InitNet(flat, 2, 3, 1, tau)
    onet_cfg = ofe.NetCfg(q, 2, 3, 1, tau)
    fe = vio.Frontend(p, w, h, 1, cap)
    fe.set_initnet(net)
    assert fe.launches_per_step() == 4
    frames = torch.from_numpy(seq.frames).cuda()
    st = ofe.StreamState()
    prev_ids = [np.zeros(0, np.int32), np.zeros(0, np.int32)]
    n_learned_o = n_learned_g = n_common = n_unconv = 0
    gate = net.cfg.max_last_step
    assert gate > 0 and onet_cfg.max_last_step == pytest.approx(gate)
    worst = 0.0
    for t in range(n_frames):
        fe.step(frames[t: t + 1])
        torch.cuda.synchronize()
        v = fe.view()
        res = ofe.step(st, seq.frames[t], op, cap, n_threads=8, net=onet_cfg)
        cnt = v["track_count"][0].cpu().numpy()
        gx = [v["track_xy"][0, c, : cnt[c]].cpu().numpy() for c in range(2)]
        gi = [v["track_id"][0, c, : cnt[c]].cpu().numpy() for c in range(2)]
        expl = set()
        for c in range(2):
            expl |= _explained_net(res["track"][c], prev_ids[c], p.fb_max_dist, tau)
            if res["track"][c] is not None:
                n_learned_o += int(res["track"][c]["learned"].sum())
        expl |= _explained(res["match"], st.ids[0][-len(res["new_xy"]):] if len(res["new_xy"])
                           else [], p.fb_max_dist)
        for c in range(2):
            gs, os_ = list(gi[c]), list(st.ids[c])
            diff = set(gs) ^ set(os_)
            assert diff <= expl, (t, c, sorted(diff - expl)[:10], len(diff))
            opos = {i: xy for i, xy in zip(os_, st.xy[c])}
            row = {i: j for j, i in enumerate(prev_ids[c])}
            for i, xy in zip(gs, gx[c]):
                if i in opos and i not in expl:
                    e = float(np.abs(np.asarray(xy, np.float64) - opos[i]).max())
                    n_common += 1
                    if e >= FLOW_TOL:
                        r = res["track"][c]
                        j = row[i]
                        assert r is not None and r["last_step"][j] > gate, (
                            t, c, i, e, r["last_step"][j], bool(r["learned"][j]))
                        n_unconv += 1
                    else:
                        worst = max(worst, e)
        stats, _ = fe.read_stats()
        n_learned_g += int(stats[t, 0, vio.STAT_NAMES.index("learned")])
        st.xy = [gx[0].copy(), gx[1].copy()]
        st.ids = [gi[0].copy(), gi[1].copy()]
        prev_ids = [gi[0].copy(), gi[1].copy()]
    assert worst < FLOW_TOL, worst
    assert n_common > 500
    assert n_unconv <= 0.01 * n_common, (n_unconv, n_common)
    assert n_learned_o > 100
    assert abs(n_learned_g - n_learned_o) <= max(3, 0.02 * n_learned_o)
    fe.close()


def test_frontend_initnet_off_is_plain():
    """Turning the initializer on with a gate nothing reaches, then off,
    gives the plain frontend's lists bit for bit."""
    w, h, L = 376, 240, 4
    seq = synth.make_sequence(5007, 4, w, h, 1, max_motion=6.0, tex_size=1024)
    p = vio.default_params(n_levels=L, cell_w=47, cell_h=40)
    cap = 2 * (w // 47) * (h // 40)
    frames = torch.from_numpy(seq.frames).cuda().view(4, 1, 2, h, w)
    flat, _ = _net_master("random")
    net = vio.InitNet(flat, 2, 3, 1, 2.0)        # confidence never reaches 2
    a, b = vio.Frontend(p, w, h, 1, cap), vio.Frontend(p, w, h, 1, cap)
    b.set_initnet(net)
    for t in range(4):
        if t == 2:
            b.set_initnet(None)
        a.step(frames[t])
        b.step(frames[t])
    torch.cuda.synchronize()
    va, vb = a.view(), b.view()
    assert torch.equal(va["track_count"], vb["track_count"])
    for c in range(2):
        n = int(va["track_count"][0, c])
        assert torch.equal(va["track_xy"][0, c, :n], vb["track_xy"][0, c, :n])
        assert torch.equal(va["track_id"][0, c, :n], vb["track_id"][0, c, :n])
    assert b.launches_per_step() == 3


def test_step_host_equals_step_and_view():
    """vio_frontend_step_host (copy in, step, copy out) gives the lists of
    vio_frontend_step read through the view."""
    w, h, L = 376, 240, 3
    seq = synth.make_sequence(5011, 4, w, h, 1, max_motion=5.0, tex_size=1024)
    p = vio.default_params(n_levels=L, cell_w=47, cell_h=40)
    cap = 2 * (w // 47) * (h // 40)
    a, b = vio.Frontend(p, w, h, 1, cap), vio.Frontend(p, w, h, 1, cap)
    host = torch.from_numpy(seq.frames).view(4, 1, 2, h, w).pin_memory()
    dev = torch.from_numpy(seq.frames).cuda().view(4, 1, 2, h, w)
    slots = torch.empty((2, 1, 2, h, w), dtype=torch.uint8, device="cuda")
    out = b.host_outputs()
    for t in range(4):
        a.step(dev[t])
        b.step_host(host[t], slots[t % 2], out)
    torch.cuda.synchronize()
    va = a.view()
    assert torch.equal(va["track_count"].cpu(), out["count"])
    for c in range(2):
        n = int(out["count"][0, c])
        assert n > 0
        assert torch.equal(va["track_xy"][0, c, :n].cpu(), out["xy"][0, c, :n])
        assert torch.equal(va["track_id"][0, c, :n].cpu(), out["id"][0, c, :n])
    nn = int(out["new_count"][0])
    assert int(va["new_count"][0]) == nn
    assert torch.equal(va["new_xy"][0, :nn].cpu(), out["new_xy"][0, :nn])


@pytest.mark.parametrize("tune", [(64, -1, 1, 128), (256, 1, 2, 256), (128, 0, 0, 128, 1),
                                  (128, 0, 0, 256, 8), (32, 0, 0, 128)])
def test_frontend_tune_does_not_change_results(tune):
    w, h, L = 376, 240, 4
    seq = synth.make_sequence(5013, 5, w, h, 1, max_motion=6.0, tex_size=1024)
    p = vio.default_params(n_levels=L, cell_w=47, cell_h=40)
    cap = 2 * (w // 47) * (h // 40)
    frames = torch.from_numpy(seq.frames).cuda().view(5, 1, 2, h, w)
    a, b = vio.Frontend(p, w, h, 1, cap), vio.Frontend(p, w, h, 1, cap)
    b.set_tune(*tune)
    a.run(frames)
    b.run(frames)
    torch.cuda.synchronize()
    va, vb = a.view(), b.view()
    assert torch.equal(va["track_count"], vb["track_count"])
    for c in range(2):
        n = int(va["track_count"][0, c])
        assert torch.equal(va["track_xy"][0, c, :n], vb["track_xy"][0, c, :n])
        assert torch.equal(va["track_id"][0, c, :n], vb["track_id"][0, c, :n])
