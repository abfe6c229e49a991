"""Learned flow initializer on the GPU against its FP64 oracle: packing and
input extraction bit for bit, the tensor-core forward pass and the training
gradient within the BF16 arithmetic's tolerance, Adam against torch.optim."""
import numpy as np
import pytest
import torch

import oracle
from oracle import initnet as onet
from paper_2609_30459_gb300 import synth

from initnet_util import GRAD_REL, KINK_MARGIN, _abs_grad, _kink_margin  # noqa: E402

pytestmark = pytest.mark.gpu

vio = pytest.importorskip("paper_2609_30459_gb300.vio")
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vio.load(build=True)
    oracle.build()


def he_params(seed):
    rng = np.random.default_rng(seed)
    fan = {"w1": 36, "w2": 288, "w3": 288, "w4": 128, "w5": 64}
    p = {}
    for k in onet.ORDER:
        if k.startswith("w"):
            p[k] = rng.normal(0, np.sqrt(2.0 / fan[k]), onet.SHAPES[k])
        else:
            p[k] = rng.normal(0, 0.05, onet.SHAPES[k])
    return p


def packed_of(flat):
    master = torch.from_numpy(flat.astype(np.float32)).to(DEV)
    packed = torch.empty(vio.INITNET_PACKED_BYTES, dtype=torch.uint8, device=DEV)
    vio.initnet_pack(master, packed)
    return master, packed


def bf16_params(flat):
    """The parameters the packed network computes with: weights BF16, biases FP32."""
    p = onet.unflatten(flat.astype(np.float32).astype(np.float64))
    return {k: (onet.bf16_round(v) if k.startswith("w") else v) for k, v in p.items()}


def bits_of(v):
    return (np.ascontiguousarray(v, np.float32).view(np.uint32) >> 16).astype(np.uint16)


def test_pack_bitexact():
    flat = onet.flatten(he_params(0))
    _, packed = packed_of(flat)
    pk = packed.cpu().numpy()
    w = pk[: 28672 * 2].view(np.uint16)
    b = pk[28672 * 2:].view(np.float32)
    p = bf16_params(flat)
    # [N][K] rows, K padded to a multiple of 16, N of the last layer to 8
    blocks = [("w1", 32, 48), ("w2", 32, 288), ("w3", 32, 288), ("w4", 64, 128), ("w5", 8, 64)]
    off = 0
    for k, n, kk in blocks:
        m = p[k].reshape(p[k].shape[0], -1)
        exp = np.zeros((n, kk))
        exp[: m.shape[0], : m.shape[1]] = m
        assert np.array_equal(w[off: off + n * kk], bits_of(exp.reshape(-1))), k
        off += n * kk
    exp_b = np.zeros(168, np.float32)
    exp_b[0:32], exp_b[32:64], exp_b[64:96] = p["b1"], p["b2"], p["b3"]
    exp_b[96:160], exp_b[160:163] = p["b4"], p["b5"]
    assert np.array_equal(b, exp_b)


def _pyramids(seed, w, h, L, n_frames=2, motion=20.0):
    seq = synth.make_sequence(seed, n_frames, w, h, 1, max_motion=motion, tex_size=1024)
    cam0 = seq.frames[:, 0]                                       # (F, h, w)
    pyr = vio.Pyramids(torch.from_numpy(np.ascontiguousarray(cam0)).to(DEV), L)
    ctx = vio.Context(vio.default_params(n_levels=L), w, h, n_frames)
    ctx.pyramid_build(pyr)
    torch.cuda.synchronize()
    return pyr, [oracle.pyramid(cam0[i], L) for i in range(n_frames)]


def _points(rng, n, w, h):
    pts = np.stack([rng.uniform(-3, w + 3, n), rng.uniform(-3, h + 3, n)], 1)
    pts[:8] = [[0, 0], [w - 1, h - 1], [0.5, 0.5], [w - 0.5, 7.49], [7.5, 7.5], [31.5, 15.5],
               [w / 2, -2.0], [100.25, 63.75]]
    return pts.astype(np.float32)


def _extract(pyr, pts, la, lb, count=None):
    n = len(pts)
    x = torch.empty((n, 4, 16, 16), dtype=torch.int16, device=DEV)
    cnt = None if count is None else torch.tensor([count], dtype=torch.int32, device=DEV)
    vio.initnet_extract(pyr, pyr.batch(0, 1, 1), pyr.batch(1, 1, 1),
                        torch.from_numpy(pts).to(DEV), cnt, n, la, lb, x)
    torch.cuda.synchronize()
    raw = x.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    return raw.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("la,lb", [(2, 3), (0, 1), (1, 1)])
def test_extract_bitexact(la, lb):
    w, h = 320, 240
    pyr, ref = _pyramids(11, w, h, 4)
    pts = _points(np.random.default_rng(la * 10 + lb), 200, w, h)
    got = _extract(pyr, pts, la, lb, count=190)
    for i in range(190):
        exp = onet.extract(ref[0], ref[1], float(pts[i, 0]), float(pts[i, 1]), la, lb)
        assert np.array_equal(got[i], exp), i
    assert np.all(got[190:] == 0.0)                    # beyond the count


def _inputs(n, seed):
    w, h = 320, 240
    pyr, _ = _pyramids(20 + seed, w, h, 4)
    rng = np.random.default_rng(seed)
    pts = np.stack([rng.uniform(8, w - 8, n), rng.uniform(8, h - 8, n)], 1).astype(np.float32)
    return _extract(pyr, pts, 2, 3)


def _forward_gpu(packed, x):
    n = len(x)
    xb = torch.from_numpy(bits_of(x.reshape(n, -1)).view(np.int16)).to(DEV)
    out = torch.empty((n, 3), dtype=torch.float32, device=DEV)
    vio.initnet_forward(packed, xb, n, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), xb


# Tolerance of the raw outputs: the GPU accumulates in FP32 in its own order,
# so a stored BF16 activation can land one BF16 step (2^-8 relative) away
# from the oracle's where the exact value sits next to a rounding boundary;
# one such step in the widest-fan-out layer moves an output by about
# |w5| * 2^-8 * |h4| ~ 1e-3. Typical differences are 1e-5.
O_TOL = 4e-3


@pytest.mark.parametrize("n", [1, 5, 333])
def test_forward_matches_oracle(n):
    flat = onet.flatten(he_params(1))
    _, packed = packed_of(flat)
    p = bf16_params(flat)
    x = _inputs(n, n)
    got, _ = _forward_gpu(packed, x)
    o = np.array([onet.forward(p, xi, act_bf16=True) for xi in x])
    exp = np.stack([o[:, 0] * 16, o[:, 1] * 16, onet.sigmoid(o[:, 2])], 1)
    err = np.abs(got - exp)
    assert np.all(err[:, :2] <= 16 * O_TOL), err.max()
    assert np.all(err[:, 2] <= O_TOL / 4)
    assert np.median(err[:, :2]) < 16 * 1e-4
    assert vio.initnet_fault() == 0           # no completion wait gave up


@pytest.mark.parametrize("radius", [1.0, 3.0])
def test_train_gradient_matches_oracle(radius):
    n = 48
    flat = onet.flatten(he_params(2))
    _, packed = packed_of(flat)
    p = bf16_params(flat)
    pool = _inputs(4 * n, 7)
    x = np.stack([xi for xi in pool if _kink_margin(p, xi) > KINK_MARGIN][:n])
    assert len(x) == n
    rng = np.random.default_rng(8)
    # targets at a chosen distance from the oracle's prediction, away from the
    # label boundary so that both sides give every sample the same label
    flows = []
    for xi in x:
        o = onet.forward(p, xi, act_bf16=True)
        r = rng.choice([rng.uniform(0.0, 0.8 * radius), rng.uniform(1.2 * radius, 6.0 * radius)])
        a = rng.uniform(0, 2 * np.pi)
        flows.append([o[0] * 16 + r * np.cos(a), o[1] * 16 + r * np.sin(a)])
    flows = np.array(flows, np.float32).astype(np.float64)
    loss_ref, g_ref = onet.batch_loss_grad(p, x, flows, act_bf16=True, radius=radius)
    g_abs = _abs_grad(p, x, flows, radius)
    xb = torch.from_numpy(bits_of(x.reshape(n, -1)).view(np.int16)).to(DEV)
    grad = torch.zeros(vio.INITNET_N_PARAMS, dtype=torch.float32, device=DEV)
    loss = torch.zeros(1, dtype=torch.float32, device=DEV)
    vio.initnet_train_step(packed, xb, torch.from_numpy(flows.astype(np.float32)).to(DEV), None,
                           n, 1.0 / n, grad, loss, label_radius=radius)
    torch.cuda.synchronize()
    assert loss.item() / n == pytest.approx(loss_ref, rel=1e-3)
    g = onet.unflatten(grad.cpu().numpy().astype(np.float64))
    for k in onet.ORDER:
        bound = GRAD_REL * g_abs[k] + 1e-7 * np.abs(g_abs[k]).max()
        err = np.abs(g[k] - g_ref[k])
        assert np.all(err <= bound), (k, float((err / np.maximum(bound, 1e-300)).max()))
        # and the typical element is far tighter than the bound
        assert np.median(err / np.maximum(g_abs[k], 1e-300)) < 1e-4, k


def test_train_index_selects_samples():
    n = 40
    flat = onet.flatten(he_params(3))
    _, packed = packed_of(flat)
    x = _inputs(n, 9)
    xb = torch.from_numpy(bits_of(x.reshape(n, -1)).view(np.int16)).to(DEV)
    flows = torch.from_numpy(np.random.default_rng(1).normal(0, 4, (n, 2)).astype(np.float32)).to(DEV)
    idx = torch.tensor([3, 17, 17, 39, 0], dtype=torch.int32, device=DEV)

    def run(xs, fl, index, m):
        grad = torch.zeros(vio.INITNET_N_PARAMS, dtype=torch.float32, device=DEV)
        loss = torch.zeros(1, dtype=torch.float32, device=DEV)
        vio.initnet_train_step(packed, xs, fl, index, m, 1.0, grad, loss)
        torch.cuda.synchronize()
        return grad.cpu().numpy(), loss.item()

    g1, l1 = run(xb, flows, idx, 5)
    sel = idx.long()
    g2, l2 = run(xb[sel].contiguous(), flows[sel].contiguous(), None, 5)
    assert l1 == pytest.approx(l2, rel=1e-5)
    assert np.allclose(g1, g2, rtol=1e-4, atol=1e-6 * np.abs(g2).max())


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(4)
    w0 = rng.normal(size=vio.INITNET_N_PARAMS).astype(np.float32)
    grads = [rng.normal(size=vio.INITNET_N_PARAMS).astype(np.float32) * s for s in (1, 0.1, 3)]
    w = torch.from_numpy(w0).to(DEV)
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    ref = torch.nn.Parameter(torch.from_numpy(w0.copy()))
    opt = torch.optim.Adam([ref], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for t, gr in enumerate(grads, start=1):
        vio.initnet_adam(w, torch.from_numpy(gr).to(DEV), m, v, t, 1e-3)
        ref.grad = torch.from_numpy(gr)
        opt.step()
    torch.cuda.synchronize()
    assert np.allclose(w.cpu().numpy(), ref.detach().numpy(), rtol=1e-5, atol=1e-6)


def test_training_reduces_loss():
    """A few hundred Adam steps on one image pair with a known shift."""
    w, h = 320, 240
    rng = np.random.default_rng(5)
    tex = synth.band_limited_texture(31, 512, 512)
    pairs, flows = [], []
    for i in range(24):
        dx, dy = rng.uniform(-12, 12, 2)
        ox, oy = rng.integers(0, 150, 2)
        # b shows a's content moved by the rounded shift: flow = that shift
        b = tex[oy - int(round(dy)) + 20: oy - int(round(dy)) + 20 + h,
                ox - int(round(dx)) + 20: ox - int(round(dx)) + 20 + w]
        a = tex[oy + 20: oy + 20 + h, ox + 20: ox + 20 + w]
        pairs.append(np.stack([synth.quantize(a, None, 0), synth.quantize(b, None, 0)]))
        flows.append((round(dx), round(dy)))
    n_per = 64
    xs, fs = [], []
    for (pa, (fx, fy)) in zip(pairs, flows):
        pyr = vio.Pyramids(torch.from_numpy(pa).to(DEV), 4)
        vio.Context(vio.default_params(n_levels=4), w, h, 2).pyramid_build(pyr)
        pts = np.stack([rng.uniform(40, w - 40, n_per), rng.uniform(40, h - 40, n_per)], 1)
        pts = pts.astype(np.float32)
        x = torch.empty((n_per, 4, 16, 16), dtype=torch.int16, device=DEV)
        vio.initnet_extract(pyr, pyr.batch(0, 1, 1), pyr.batch(1, 1, 1),
                            torch.from_numpy(pts).to(DEV), None, n_per, 2, 3, x)
        xs.append(x)
        fs.append(torch.tensor([[fx, fy]] * n_per, dtype=torch.float32, device=DEV))
    X = torch.cat(xs)
    F = torch.cat(fs)
    N = len(X)
    master = torch.from_numpy(onet.flatten(he_params(6)).astype(np.float32)).to(DEV)
    packed = torch.empty(vio.INITNET_PACKED_BYTES, dtype=torch.uint8, device=DEV)
    m, v = torch.zeros_like(master), torch.zeros_like(master)
    grad = torch.zeros_like(master)
    loss = torch.zeros(1, dtype=torch.float32, device=DEV)
    hist = []
    gen = torch.Generator(device="cpu").manual_seed(0)
    for step in range(1, 301):
        idx = torch.randperm(N, generator=gen)[:256].to(torch.int32).to(DEV)
        vio.initnet_pack(master, packed)
        grad.zero_()
        loss.zero_()
        vio.initnet_train_step(packed, X, F, idx, 256, 1.0 / 256, grad, loss)
        vio.initnet_adam(master, grad, m, v, step, 2e-3)
        if step <= 10 or step > 290:
            hist.append(loss.item() / 256)
    assert np.mean(hist[-10:]) < np.mean(hist[:10]), hist
    # the flow itself: the trained proposals are far closer than a zero start
    vio.initnet_pack(master, packed)
    out = torch.empty((N, 3), dtype=torch.float32, device=DEV)
    vio.initnet_forward(packed, X, N, out)
    err = torch.linalg.norm(out[:, :2] - F, dim=1)
    zero = torch.linalg.norm(F, dim=1)
    assert err.median().item() < 0.3 * zero.median().item(), (err.median(), zero.median())


def test_checkpoint_save_load_resume(tmp_path):
    """Weights, Adam moments, step count and gate configuration survive a
    save/load; training resumes from the loaded state."""
    flat = onet.flatten(he_params(8)).astype(np.float32)
    net = vio.InitNet(flat, 2, 3, 1, 0.4)
    x = _inputs(64, 3)
    xb = torch.from_numpy(bits_of(x.reshape(64, -1)).view(np.int16)).to(DEV)
    flows = torch.from_numpy(np.random.default_rng(2).normal(0, 4, (64, 2)).astype(np.float32)).to(DEV)
    from paper_2609_30459_gb300 import initnet_train
    initnet_train.train(net, xb, flows, epochs=1, batch=32, lr=1e-3, log=lambda *_: None)
    path = tmp_path / "ck.npz"
    net.save(path, label_radius=3.0)
    back = vio.InitNet.load(path)
    assert back.step == net.step == 2
    assert torch.equal(back.master, net.master) and torch.equal(back.m, net.m)
    assert torch.equal(back.v, net.v)
    assert (back.cfg.level_a, back.cfg.level_b, back.cfg.start_level) == (2, 3, 1)
    assert back.cfg.min_conf == pytest.approx(0.4)
    assert torch.equal(back.packed, net.packed)
    # one more epoch from either copy: the same update (up to the order of
    # the floating-point gradient sums)
    initnet_train.train(net, xb, flows, epochs=1, batch=32, lr=1e-3, log=lambda *_: None)
    initnet_train.train(back, xb, flows, epochs=1, batch=32, lr=1e-3, log=lambda *_: None)
    assert back.step == net.step == 4
    assert torch.allclose(back.master, net.master, rtol=1e-4, atol=1e-6)
