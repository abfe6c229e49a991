"""Pins of the learned initializer's FP64 oracle: the convolution against a
library correlation, analytic gradients against central finite differences,
and the loss gradient in closed form. No GPU."""
import numpy as np
import pytest
from scipy import signal

from oracle import initnet as net


def rand_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return {k: rng.normal(0, scale, net.SHAPES[k]) for k in net.ORDER}


def test_conv_matches_library_correlation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(4, 16, 16))
    w = rng.normal(size=(5, 4, 3, 3))
    b = rng.normal(size=5)
    got = net.conv_s2(x, w, b)
    for o in range(5):
        full = sum(signal.correlate2d(np.pad(x[c], 1), w[o, c], mode="valid") for c in range(4))
        assert np.allclose(got[o], full[::2, ::2] + b[o], atol=1e-12)


def test_shapes_and_param_count():
    p = rand_params(1)
    o = net.forward(p, np.zeros((4, 16, 16)))
    assert o.shape == (3,)
    assert net.n_params() == 32 * 36 + 32 + 2 * (32 * 288 + 32) + 64 * 128 + 64 + 3 * 64 + 3
    assert np.array_equal(net.flatten(net.unflatten(net.flatten(p))), net.flatten(p))


def test_loss_gradient_closed_form():
    o = np.array([0.2, -0.1, 0.3])
    flow = np.array([2.0, -3.0])
    loss, do = net.loss_and_grad_out(o, flow)
    s = 1 / (1 + np.exp(-0.3))
    # predicted flow (3.2, -1.6) is more than 1 px from (2, -3): label 0
    assert do[0] == pytest.approx(2 * (0.2 - 2 / 16)) and do[1] == pytest.approx(2 * (-0.1 + 3 / 16))
    assert do[2] == pytest.approx(s)
    assert loss == pytest.approx((0.2 - 0.125) ** 2 + (-0.1 + 0.1875) ** 2 - np.log(1 - s))


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    p = rand_params(seed + 10, scale=0.1)
    # inputs whose pre-activations all stay 1e-3 away from the ReLU kinks, so
    # that a step of 1e-5 in one weight cannot cross one
    xs, flows = [], []
    while len(xs) < 2:
        x = rng.normal(size=(4, 16, 16))
        f = rng.normal(0, 4, size=2)
        o, act = net.forward(p, x, keep=True)
        margin = min(np.abs(act[k]).min() for k in ("a1", "a2", "a3", "a4"))
        dist = np.hypot(o[0] * net.SCALE - f[0], o[1] * net.SCALE - f[1])
        if margin > 1e-3 and abs(dist - 1.0) > 1e-2:
            xs.append(x)
            flows.append(f)
    xs, flows = np.array(xs), np.array(flows)
    _, g = net.batch_loss_grad(p, xs, flows)
    flat = net.flatten(p)
    gflat = net.flatten(g)
    idx = rng.choice(len(flat), 60, replace=False)
    idx = np.concatenate([idx, [0, len(flat) - 1, net.n_params() - 3 * 64 - 3]])

    def f(v):
        return net.batch_loss_grad(net.unflatten(v), xs, flows)[0]

    # a central difference is exact to O(h^2) away from ReLU kinks and label
    # flips; a wrong sign or index would be off by O(1), not 1e-3
    h = 1e-5
    for i in idx:
        vp, vm = flat.copy(), flat.copy()
        vp[i] += h
        vm[i] -= h
        fd = (f(vp) - f(vm)) / (2 * h)
        assert fd == pytest.approx(gflat[i], rel=1e-3, abs=1e-6), i


def test_extract_samples_integer_grid():
    src = [np.arange(64 * 64, dtype=np.int64).reshape(64, 64) % 256,
           np.full((32, 32), 192)]
    dst = [np.full((64, 64), 128), np.full((32, 32), 64)]
    x = net.extract(src, dst, 20.4, 30.6, 0, 1)
    # level 0 window starts at round(20.4)-8 = 12, round(30.6)-8 = 23
    assert x[0, 0, 0] == ((23 * 64 + 12) % 256 - 128) / 64
    assert np.all(x[1] == 0.0) and np.all(x[2] == 1.0) and np.all(x[3] == -1.0)


def test_bf16_round_special_values_and_library():
    import torch
    # exact values stay, ties go to the even neighbour, halfway+ goes up
    assert net.bf16_round([1.0, -2.5, 0.0])[0] == 1.0
    assert net.bf16_round([1 + 2 ** -8])[0] == 1.0                    # tie, 1.0 is even
    assert net.bf16_round([1 + 3 * 2 ** -8])[0] == 1 + 2 ** -6        # tie, rounds up to even
    assert net.bf16_round([1 + 2 ** -8 + 2 ** -20])[0] == 1 + 2 ** -7
    rng = np.random.default_rng(3)
    v = (rng.normal(size=4096) * 10.0 ** rng.integers(-6, 6, 4096)).astype(np.float32)
    lib = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(net.bf16_round(v), lib)


def test_bf16_activations_only_round_the_stored_values():
    p = {k: net.bf16_round(v) for k, v in rand_params(4, 0.2).items()}
    x = net.bf16_round(np.random.default_rng(5).normal(size=(4, 16, 16)))
    o64 = net.forward(p, x)
    o16, act = net.forward(p, x, keep=True, act_bf16=True)
    for k in ("h1", "h2", "h3", "h4"):
        assert np.array_equal(net.bf16_round(act[k]), act[k])
    # BF16 storage perturbs each activation by at most 2^-9 relative
    assert np.max(np.abs(o16 - o64)) < 0.05 * (1 + np.max(np.abs(o64)))


def test_label_radius_sets_the_confidence_target():
    o = np.array([0.2, -0.1, 0.3])
    flow = np.array([2.0, -3.0])              # about 1.8 px from the prediction (3.2, -1.6)
    d = np.hypot(0.2 * 16 - 2.0, -0.1 * 16 + 3.0)
    s = 1 / (1 + np.exp(-0.3))
    _, do_in = net.loss_and_grad_out(o, flow, radius=d + 0.01)
    _, do_out = net.loss_and_grad_out(o, flow, radius=d - 0.01)
    assert do_in[2] == pytest.approx(s - 1) and do_out[2] == pytest.approx(s)
    assert do_in[0] == do_out[0] and do_in[1] == do_out[1]
