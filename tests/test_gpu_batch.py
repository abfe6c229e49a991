"""Batched multi-stream frontend (mixed sizes, per-stream state, graph
replay, autotuner): every stream's result in the batch equals the same
stream run alone through vio_frontend on the same frames, bit for bit."""
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


GROUPS = [  # w, h, n_streams, cell, levels
    (376, 240, 2, 37, 4),
    (320, 256, 3, 40, 3),
]
N_FRAMES = 5


def _make():
    seqs, groups = [], []
    for gi, (w, h, n, cell, L) in enumerate(GROUPS):
        p = vio.default_params(n_levels=L, cell_w=cell, cell_h=cell)
        cap = 2 * (w // cell) * (h // cell)
        groups.append((p, w, h, n, cap))
        seqs.append([synth.make_sequence(6000 + 10 * gi + s, N_FRAMES, w, h, 1,
                                         max_motion=6.0, tex_size=1024).frames
                     for s in range(n)])
    return groups, seqs


def _alone(p, w, h, cap, frames, steps, net=None):
    """Lists of one stream run alone over frames[t] for t in steps."""
    fe = vio.Frontend(p, w, h, 1, cap)
    if net is not None:
        fe.set_initnet(net)
    keep = []
    for t in steps:
        f = torch.from_numpy(frames[t]).cuda().view(1, 2, h, w)
        keep.append(f)
        fe.step(f)
    torch.cuda.synchronize()
    v = fe.view()
    cnt = v["track_count"][0].cpu().numpy()
    out = ([v["track_xy"][0, c, : cnt[c]].cpu().numpy() for c in range(2)],
           [v["track_id"][0, c, : cnt[c]].cpu().numpy() for c in range(2)])
    fe.close()
    return out


def _run_batch(b, seqs, schedule, stream=None):
    """schedule: list of activity lists (one flag per stream, groups in order)."""
    t_of = [[0] * len(g) for g in seqs]
    for act in schedule:
        k = 0
        for gi, g in enumerate(seqs):
            for s in range(len(g)):
                if act[k]:
                    b.next_frame(gi, s).copy_(torch.from_numpy(g[s][t_of[gi][s]]).cuda())
                    t_of[gi][s] += 1
                k += 1
        b.step(act, stream=stream)
    torch.cuda.synchronize()


def _check_equal(b, groups, seqs, schedule, net=None):
    k = 0
    for gi, (p, w, h, n, cap) in enumerate(groups):
        for s in range(n):
            steps = [i for i, act in enumerate(schedule) if act[k]]
            ref_xy, ref_id = _alone(p, w, h, cap, seqs[gi][s], range(len(steps)), net)
            xy, ids = b.stream_lists(gi, s)
            for c in range(2):
                assert np.array_equal(ids[c], ref_id[c]), (gi, s, c)
                assert np.array_equal(xy[c], ref_xy[c]), (gi, s, c)
            assert len(ids[0]) > 0
            k += 1


def test_batch_equals_streams_alone():
    groups, seqs = _make()
    b = vio.Batch(groups)
    total = sum(g[3] for g in groups)
    schedule = [[1] * total for _ in range(N_FRAMES)]
    _run_batch(b, seqs, schedule)
    _check_equal(b, groups, seqs, schedule)


def test_batch_skipped_streams_keep_their_state():
    groups, seqs = _make()
    b = vio.Batch(groups)
    rng = np.random.default_rng(0)
    total = sum(g[3] for g in groups)
    schedule = [[1] * total] + [list((rng.random(total) < 0.6).astype(int)) for _ in range(6)]
    # at most N_FRAMES active steps per stream
    for k in range(total):
        n_act = 0
        for act in schedule:
            if act[k]:
                n_act += 1
                if n_act > N_FRAMES:
                    act[k] = 0
    _run_batch(b, seqs, schedule)
    _check_equal(b, groups, seqs, schedule)


def test_batch_graph_replay_and_autotune():
    groups, seqs = _make()
    total = sum(g[3] for g in groups)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = vio.Batch(groups)
        # frames in both slots for the autotuner
        for gi, g in enumerate(seqs):
            for st in range(len(g)):
                for t in range(2):
                    b.next_frame(gi, st).copy_(torch.from_numpy(g[st][t]).cuda())
                    b.step([1 if (i == sum(x[3] for x in groups[:gi]) + st) else 0
                            for i in range(total)], stream=s)
        best = b.autotune(reps=1, stream=s)
        assert best > 0
        k2, shift, after, first, k1, dw = b.get_tune()
        assert k2 in (32, 64, 128, 256, 512) and shift in (-1, 0, 1) and after in (0, 1)
        assert first in (0, 1, 2) and k1 in (128, 256)
        b.set_graph(True)
        schedule = [[1] * total for _ in range(N_FRAMES)]
        _run_batch(b, seqs, schedule, stream=s)
    s.synchronize()
    _check_equal(b, groups, seqs, schedule)
    assert b.launches_per_step() >= 3 + 2 * after


@pytest.mark.parametrize("first", [1, 2])
def test_batch_pyramid_split_equals_streams_alone(first):
    """Fewer levels in the fused pyramid+detection launch (the rest in
    further pyramid launches) gives the same lists."""
    groups, seqs = _make()
    total = sum(g[3] for g in groups)
    b = vio.Batch(groups)
    b.set_tune(256, 1, 0, first, 128, 2)
    assert b.get_tune() == (256, 1, 0, first, 128, 2)
    schedule = [[1] * total for _ in range(N_FRAMES)]
    _run_batch(b, seqs, schedule)
    _check_equal(b, groups, seqs, schedule)
    # 4 levels (group 0) and 3 (group 1): one more pyramid launch per group
    # whose levels do not all fit in the first pass
    assert b.launches_per_step() == 3 + (2 if first == 1 else 1)


@pytest.mark.parametrize("learned", [False, True])
def test_batch_stereo_after_selection_equals_streams_alone(learned):
    """Matching only the selected keypoints, after selection, gives the same
    lists as the frontend's order (every candidate matched beside temporal
    tracking), with and without the learned start, skipped streams included."""
    groups, seqs = _make()
    net = None
    if learned:
        rng = np.random.default_rng(5)
        flat = (rng.normal(0, 0.05, vio.INITNET_N_PARAMS)).astype(np.float32)
        flat[-1] = 3.0
        net = vio.InitNet(flat, 1, 2, 1, 0.5)
    total = sum(g[3] for g in groups)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = vio.Batch(groups)
        if net is not None:
            b.set_initnet(net)
        b.set_tune(128, 0, 1)
        b.set_graph(True)
        assert b.launches_per_step() == (4 if learned else 3) + 2
        rng2 = np.random.default_rng(2)
        schedule = [[1] * total] + [list((rng2.random(total) < 0.7).astype(int))
                                    for _ in range(5)]
        for k in range(total):
            n_act = 0
            for act in schedule:
                if act[k]:
                    n_act += 1
                    if n_act > N_FRAMES:
                        act[k] = 0
        _run_batch(b, seqs, schedule, stream=s)
    s.synchronize()
    _check_equal(b, groups, seqs, schedule, net)


def test_batch_with_initnet_equals_streams_alone():
    """With the learned start on (every group, graphs on), each stream's lists
    equal the same stream alone through vio_frontend with the same network."""
    groups, seqs = _make()
    rng = np.random.default_rng(3)
    flat = (rng.normal(0, 0.05, vio.INITNET_N_PARAMS)).astype(np.float32)
    flat[-1] = 3.0                                   # confident proposals
    net = vio.InitNet(flat, 1, 2, 1, 0.5)
    total = sum(g[3] for g in groups)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = vio.Batch(groups)
        b.set_initnet(net)
        b.set_graph(True)
        assert b.launches_per_step() == 4
        rng2 = np.random.default_rng(1)
        schedule = [[1] * total] + [list((rng2.random(total) < 0.7).astype(int))
                                    for _ in range(5)]
        for k in range(total):
            n_act = 0
            for act in schedule:
                if act[k]:
                    n_act += 1
                    if n_act > N_FRAMES:
                        act[k] = 0
        _run_batch(b, seqs, schedule, stream=s)
    s.synchronize()
    _check_equal(b, groups, seqs, schedule, net)


@pytest.mark.parametrize("learned", [False, True])
def test_batch_filling_the_gpu_equals_streams_alone(learned):
    """A batch with more keypoints than 16 per SM tracks them with the
    reduction form for launches that fill the GPU; a stream alone is a small
    launch, tracked with the other form (trk::warp_sum4): the lists agree bit
    for bit, the learned start's kept and rejected first passes included."""
    w, h, cell, L = 376, 240, 37, 4
    cells = (w // cell) * (h // cell)
    cap = 2 * cells
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 16 * sms // (2 * cap + cells) + 1
    p = vio.default_params(n_levels=L, cell_w=cell, cell_h=cell)
    groups = [(p, w, h, n, cap)]
    seqs = [[synth.make_sequence(6100 + s, N_FRAMES, w, h, 1, max_motion=6.0,
                                 tex_size=1024).frames for s in range(n)]]
    net = None
    if learned:
        rng = np.random.default_rng(7)
        flat = (rng.normal(0, 0.05, vio.INITNET_N_PARAMS)).astype(np.float32)
        flat[-1] = 3.0                               # confident proposals
        net = vio.InitNet(flat, 1, 2, 1, 0.5)
    b = vio.Batch(groups)
    if net is not None:
        b.set_initnet(net)
    schedule = [[1] * n for _ in range(N_FRAMES)]
    _run_batch(b, seqs, schedule)
    _check_equal(b, groups, seqs, schedule, net)
