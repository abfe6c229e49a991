"""The multi-rank path of the benchmark on CPU ranks (gloo, world size 2):
each rank runs its own sequence, the job's time is the slowest rank's, and
the barrier and reductions work without a GPU."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2609_30459_gb300 import synth
    t = 0.5 + rank                                   # this rank's "time"
    dist.barrier()
    t_max = bench.max_over_ranks(t, dist, "cpu")
    seed = bench.seq_seed(rank)
    frames = synth.make_sequence(seed, 2, 64, 48, 1, max_motion=3.0, tex_size=256).frames
    q.put((rank, t_max, seed, frames.sum(dtype=np.int64)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, f0), (r1, t1, s1, f1) = res
    assert t0 == t1 == pytest.approx(1.5)            # max over ranks, same on both
    assert s0 != s1 and f0 != f1                      # independent sequences per rank


def test_single_process_max_is_identity():
    import bench
    assert bench.max_over_ranks(2.5, None) == 2.5
