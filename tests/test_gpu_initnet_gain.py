"""What the trained initializer gains over the plain tracker (the shipped
weights, held-out sequences with motion up to 40 px, 5 levels): the plain
pyramidal KLT from a zero start is the yardstick. A learned track counts only
when it ends OK and has converged (its last level-0 step within the network's
gate), so where the plain result ends OK and has converged too, the two agree
within 1e-3 px (>= 99.9%), and where the plain result ends OK at all nearly
always; the learned start must track over fewer levels; and the tracks it
keeps that the plain tracker loses must be right (ground truth of the
generator)."""
import os

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


def test_trained_initializer_gain():
    from paper_2609_30459_gb300 import initnet_train as it
    assert os.path.exists(it.DEFAULT_WEIGHTS), "shipped weights missing"
    net = vio.InitNet.load(it.DEFAULT_WEIGHTS)
    seqs = [synth.make_sequence(7000 + i, 12, 640, 480, 1, max_motion=40.0, tex_size=2048)
            for i in range(2)]
    g = it.gain_eval(net, seqs, n_levels=5, cell=32, start_levels=(net.cfg.start_level,),
                     taus=(net.cfg.min_conf,))
    r = g[f"start{net.cfg.start_level}_tau{net.cfg.min_conf}"]
    print(g)
    assert g["n"] > 5000
    assert r["gated"] > 0.3                         # the gate lets a good share through
    assert r["learned_ok_of_gated"] > 0.85          # and those mostly end OK and converged
    assert r["agree_of_both_ok"] > 0.99             # at the plain result within 1e-3 px,
    assert r["agree_where_plain_converged"] >= 0.999   # and wherever the plain result is
    assert r["plain_converged_of_both_ok"] > 0.95      # settled (converged) too
    assert r["levels_per_kp"] < 0.85 * g["n_levels"]
    assert r["plain_ok_within_truth"] > 0.95
    assert r["gained"] >= 0
    if r["gained"] > 50:
        assert r["gained_within_truth"] > 0.9
