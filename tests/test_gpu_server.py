"""Serving loop (vio_server): sessions served by continuous batching give,
frame by frame, the results of the same stream run alone through
vio_frontend; sessions beyond the memory budget wait for a slot and are then
served the same way."""
import numpy as np
import pytest
import torch

from paper_2609_30459_gb300 import serving, synth

pytestmark = pytest.mark.gpu

vio = pytest.importorskip("paper_2609_30459_gb300.vio")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vio.load(build=True)


CLASSES = [(320, 240, 40, 3), (376, 240, 47, 4)]     # w, h, cell, levels
N_FRAMES = 5


def _classes(n_sessions):
    out = []
    for (w, h, cell, L) in CLASSES:
        p = vio.default_params(n_levels=L, cell_w=cell, cell_h=cell)
        out.append((p, w, h, n_sessions, 2 * (w // cell) * (h // cell)))
    return out


def _frames(cls, i):
    w, h = CLASSES[cls][:2]
    f = synth.make_sequence(8000 + 10 * cls + i, N_FRAMES, w, h, 1, max_motion=6.0,
                            tex_size=1024).frames
    return torch.from_numpy(f).pin_memory()                    # (F, 2, h, w) pinned


def _alone(cl, frames, net=None):
    p, w, h, _, cap = cl
    fe = vio.Frontend(p, w, h, 1, cap)
    if net is not None:
        fe.set_initnet(net)
    counts, keep = [], []
    for t in range(len(frames)):
        f = frames[t].cuda().view(1, 2, h, w)
        keep.append(f)
        fe.step(f)
        torch.cuda.synchronize()
        counts.append(fe.view()["track_count"][0].cpu().numpy().copy())
    v = fe.view()
    lists = [(v["track_xy"][0, c, : counts[-1][c]].cpu().numpy(),
              v["track_id"][0, c, : counts[-1][c]].cpu().numpy()) for c in range(2)]
    fe.close()
    return np.array(counts), lists


def _serve(srv, sessions, trace, frames, timeout=120.0):
    reqs = []
    for (t, i, k) in trace:
        sid = sessions[i]
        flags = vio.SERVER_LAST if k == N_FRAMES - 1 else 0
        reqs.append((sid, t, frames[i][k], k, flags))
    return srv.run_trace(reqs, timeout_s=timeout)


def _check(done, sessions, outs, cls_of, frames, cl, net=None):
    assert (done["status"] == 0).all()
    for i, sid in enumerate(sessions):
        mine = np.sort(done[done["session"] == sid], order="tag")
        assert list(mine["tag"]) == list(range(N_FRAMES))
        counts, lists = _alone(cl[cls_of[i]], frames[i], net)
        got = np.stack([mine["n_tracks0"], mine["n_tracks1"]], 1)
        assert np.array_equal(got, counts), (i, got, counts)
        xy, ids, cnt = outs[i]
        assert np.array_equal(cnt, counts[-1])
        for c in range(2):
            n = counts[-1][c]
            assert np.array_equal(xy[c, :n], lists[c][0]), (i, c)
            assert np.array_equal(ids[c, :n], lists[c][1]), (i, c)
        assert counts[-1].sum() > 0


@pytest.mark.parametrize("learned", [False, True])
def test_served_sessions_equal_streams_alone(learned):
    cl = _classes(3)
    srv = vio.Server(cl, 1 << 34)
    net = None
    if learned:
        rng = np.random.default_rng(3)
        flat = rng.normal(0, 0.05, vio.INITNET_N_PARAMS).astype(np.float32)
        flat[-1] = 3.0
        net = vio.InitNet(flat, 1, 2, 1, 0.5)
        srv.set_initnet(net)
    sessions, outs, cls_of, frames = [], [], [], []
    for c in range(len(CLASSES)):
        for i in range(3):
            sid, adm = srv.open(c)
            assert adm
            cap = cl[c][4]
            out = (np.zeros((2, cap, 2), np.float32), np.zeros((2, cap), np.int32),
                   np.zeros(2, np.int32))
            srv.set_output(sid, *out)
            sessions.append(sid)
            outs.append(out)
            cls_of.append(c)
            frames.append(_frames(c, i))
    rates = np.random.default_rng(1).uniform(30, 200, len(sessions))
    trace = serving.poisson_trace(rates, 10.0, seed=2, max_frames=[N_FRAMES] * len(sessions))
    done, steps = _serve(srv, sessions, trace, frames)
    assert len(done) == N_FRAMES * len(sessions)
    assert steps <= len(done)
    _check(done, sessions, outs, cls_of, frames, cl, net)
    s = serving.latency_summary(done)
    assert s["failed"] == 0 and s["p99_ms"] > 0
    srv.close_server()


def test_admission_waits_for_a_slot():
    one, _ = vio.server_plan(_classes(1), 1 << 34)
    _, bytes1 = vio.server_plan(_classes(1), 1 << 34)
    cl = _classes(3)
    slots, _ = vio.server_plan(cl, bytes1 + 1024)
    assert slots == [1, 1]
    srv = vio.Server(cl, bytes1 + 1024)
    assert srv.slots(0)[0] == 1 and srv.slots(1)[0] == 1
    sessions, outs, cls_of, frames, admitted = [], [], [], [], []
    for c in range(len(CLASSES)):
        for i in range(3):
            sid, adm = srv.open(c)
            admitted.append(adm)
            cap = cl[c][4]
            out = (np.zeros((2, cap, 2), np.float32), np.zeros((2, cap), np.int32),
                   np.zeros(2, np.int32))
            srv.set_output(sid, *out)
            sessions.append(sid)
            outs.append(out)
            cls_of.append(c)
            frames.append(_frames(c, i))
    assert admitted == [True, False, False, True, False, False]
    # every session sends its frames at once, early: the waiting ones queue
    trace = sorted(((0.001 * k + 0.0001 * i, i, k) for i in range(len(sessions))
                    for k in range(N_FRAMES)), key=lambda r: (r[0], r[1]))
    done, _ = _serve(srv, sessions, trace, frames)
    assert len(done) == N_FRAMES * len(sessions)
    _check(done, sessions, outs, cls_of, frames, cl)
    # per class, a session starts only after the previous one has finished
    for c in range(len(CLASSES)):
        sids = [s for s, k in zip(sessions, cls_of) if k == c]
        for a, b in zip(sids, sids[1:]):
            last_a = done[done["session"] == a]["t_done"].max()
            first_b = done[done["session"] == b]["t_launch"].min()
            assert first_b >= last_a
    srv.close_server()


def test_server_rejects_bad_requests_on_the_host():
    """Failures are reported on the host before anything is enqueued: an
    unknown session, a frame after the session's last, a missing frame; a
    waiting session that closes leaves the queue without running."""
    cl = _classes(2)
    slots, _ = vio.server_plan(_classes(1), 1 << 34)
    _, bytes1 = vio.server_plan(_classes(1), 1 << 34)
    srv = vio.Server(cl, bytes1 + 1024)               # one slot per class
    a, adm_a = srv.open(0)
    b, adm_b = srv.open(0)
    assert adm_a and not adm_b
    fr = _frames(0, 0)
    with pytest.raises(vio.VioError):
        srv.submit(12345, fr[0], vio.server_now(), 0)
    srv.submit(a, fr[0], vio.server_now(), 0, vio.SERVER_LAST)
    with pytest.raises(vio.VioError):
        srv.submit(a, fr[1], vio.server_now(), 1)      # after its last frame
    srv.close(b)                                        # waiting: leaves the queue
    with pytest.raises(vio.VioError):
        srv.submit(b, fr[0], vio.server_now(), 0)
    done = []
    t0 = vio.server_now()
    while len(done) < 1 and vio.server_now() - t0 < 30:
        srv.poll()
        done.extend(srv.take())
    assert len(done) == 1 and done[0]["session"] == a and done[0]["status"] == 0
    # the slot is free again: a new session is admitted at once
    c, adm_c = srv.open(0)
    assert adm_c
    srv.close_server()
