"""Oracle of the learned flow initializer. TEST INFRASTRUCTURE ONLY.

The paper has no learned component (its initialisation projects through the
camera model, Sec. III-E); this network is an addition whose definition the
oracle states plainly, in FP64, for the GPU forward and gradient checks:

* input x: 4 channels of 16 x 16 -- source and target patch at pyramid level
  a, then source and target at level b, sampled on the integer grid around
  the keypoint and scaled as (v - 128) / 64;
* conv1 4->32, conv2 32->32, conv3 32->32: 3x3, stride 2, zero padding 1,
  ReLU after each (16x16 -> 8x8 -> 4x4 -> 2x2);
* flatten (channel, row, column) -> 128; fc1 128->64 + ReLU; fc2 64->3;
* outputs: flow = (o0, o1) * S (S = 16 px, level-0 pixels), confidence =
  sigmoid(o2);
* loss per sample: (o0 - fx/S)^2 + (o1 - fy/S)^2 + BCE(sigmoid(o2), y) with
  y = 1 if the predicted flow is within r px of the target (r = the label
  radius, 1 px unless set; y carries no gradient); the batch loss is the
  mean.

Precision: the network's weights and inputs are BF16 values and its
activations are stored as BF16 between layers (accumulation wider). The
oracle computes in FP64 on weights the caller rounds with ``bf16_round``;
``forward(..., act_bf16=True)`` also rounds each stored activation to BF16, so
that decisions taken on the outputs (the confidence gate) are taken in the
network's own precision.
"""
from __future__ import annotations

import numpy as np

SCALE = 16.0
SHAPES = {"w1": (32, 4, 3, 3), "b1": (32,), "w2": (32, 32, 3, 3), "b2": (32,),
          "w3": (32, 32, 3, 3), "b3": (32,), "w4": (64, 128), "b4": (64,),
          "w5": (3, 64), "b5": (3,)}
ORDER = ("w1", "b1", "w2", "b2", "w3", "b3", "w4", "b4", "w5", "b5")


def n_params() -> int:
    return sum(int(np.prod(SHAPES[k])) for k in ORDER)


def unflatten(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = np.asarray(flat[o:o + n], np.float64).reshape(SHAPES[k])
        o += n
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], np.float64).reshape(-1) for k in ORDER])


def bf16_round(a) -> np.ndarray:
    """Nearest BF16 value (ties to even) of each element, via float32: BF16 is
    the upper 16 bits of an IEEE binary32, so rounding adds 0x7fff plus the
    lowest kept bit to the bit pattern and clears the low 16 bits."""
    f = np.ascontiguousarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv_s2(x, w, b):
    """out[o,i,j] = b[o] + sum_{c,u,v} w[o,c,u,v] x[c, 2i+u-1, 2j+v-1], zero padded."""
    C, H, W = x.shape
    O = w.shape[0]
    Ho, Wo = H // 2, W // 2
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((O, Ho, Wo))
    for i in range(Ho):
        for j in range(Wo):
            patch = xp[:, 2 * i:2 * i + 3, 2 * j:2 * j + 3]          # (C, 3, 3)
            out[:, i, j] = b + np.tensordot(w, patch, axes=([1, 2, 3], [0, 1, 2]))
    return out


def conv_s2_backward(x, w, dout):
    """Gradients of conv_s2 w.r.t. x, w, b."""
    C, H, W = x.shape
    O, Ho, Wo = dout.shape
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for i in range(Ho):
        for j in range(Wo):
            patch = xp[:, 2 * i:2 * i + 3, 2 * j:2 * j + 3]
            g = dout[:, i, j]                                      # (O,)
            dw += g[:, None, None, None] * patch[None]
            dxp[:, 2 * i:2 * i + 3, 2 * j:2 * j + 3] += np.tensordot(g, w, axes=(0, 0))
    return dxp[:, 1:-1, 1:-1], dw, dout.sum(axis=(1, 2))


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(p: dict, x: np.ndarray, keep: bool = False, act_bf16: bool = False):
    """x: (4, 16, 16). Returns o (3,) and, if keep, the activations."""
    q = bf16_round if act_bf16 else (lambda v: v)
    a1 = conv_s2(x, p["w1"], p["b1"])
    h1 = q(np.maximum(a1, 0))
    a2 = conv_s2(h1, p["w2"], p["b2"])
    h2 = q(np.maximum(a2, 0))
    a3 = conv_s2(h2, p["w3"], p["b3"])
    h3 = q(np.maximum(a3, 0))
    f = h3.reshape(-1)
    a4 = p["w4"] @ f + p["b4"]
    h4 = q(np.maximum(a4, 0))
    o = p["w5"] @ h4 + p["b5"]
    if keep:
        return o, dict(x=x, a1=a1, h1=h1, a2=a2, h2=h2, a3=a3, h3=h3, f=f, a4=a4, h4=h4)
    return o


def outputs(o):
    """(flow dx, flow dy, confidence) from the raw outputs."""
    return o[0] * SCALE, o[1] * SCALE, sigmoid(o[2])


def loss_and_grad_out(o, flow, radius=1.0):
    """Loss of one sample and dL/do (the label carries no gradient)."""
    t0, t1 = flow[0] / SCALE, flow[1] / SCALE
    y = 1.0 if np.hypot(o[0] * SCALE - flow[0], o[1] * SCALE - flow[1]) < radius else 0.0
    s = sigmoid(o[2])
    eps = 1e-12
    loss = (o[0] - t0) ** 2 + (o[1] - t1) ** 2 - (y * np.log(s + eps) +
                                                   (1 - y) * np.log(1 - s + eps))
    do = np.array([2 * (o[0] - t0), 2 * (o[1] - t1), s - y])
    return loss, do


def backward(p: dict, act: dict, do: np.ndarray) -> dict:
    g = {}
    g["w5"] = np.outer(do, act["h4"])
    g["b5"] = do.copy()
    dh4 = p["w5"].T @ do
    da4 = dh4 * (act["a4"] > 0)
    g["w4"] = np.outer(da4, act["f"])
    g["b4"] = da4
    df = p["w4"].T @ da4
    da3 = df.reshape(act["a3"].shape) * (act["a3"] > 0)
    dh2, g["w3"], g["b3"] = conv_s2_backward(act["h2"], p["w3"], da3)
    da2 = dh2 * (act["a2"] > 0)
    dh1, g["w2"], g["b2"] = conv_s2_backward(act["h1"], p["w2"], da2)
    da1 = dh1 * (act["a1"] > 0)
    _, g["w1"], g["b1"] = conv_s2_backward(act["x"], p["w1"], da1)
    return g


def batch_loss_grad(p: dict, xs: np.ndarray, flows: np.ndarray, act_bf16: bool = False,
                    radius: float = 1.0):
    """Mean loss and gradient (dict) over a batch."""
    total = 0.0
    acc = {k: np.zeros(SHAPES[k]) for k in ORDER}
    for x, f in zip(xs, flows):
        o, act = forward(p, x, keep=True, act_bf16=act_bf16)
        loss, do = loss_and_grad_out(o, f, radius)
        total += loss
        g = backward(p, act, do)
        for k in ORDER:
            acc[k] += g[k]
    n = len(xs)
    return total / n, {k: v / n for k, v in acc.items()}


def extract(src_levels, dst_levels, px: float, py: float, la: int, lb: int) -> np.ndarray:
    """Network input of keypoint (px, py) (level-0 px): for level l in (la, lb),
    the 16 x 16 integer grid starting at round(p / 2^l) - 8 in the source and
    the target (identity position), values (v - 128) / 64, 0 outside."""
    x = np.zeros((4, 16, 16))
    for ch, (lv, img) in enumerate(((la, src_levels), (la, dst_levels),
                                    (lb, src_levels), (lb, dst_levels))):
        im = np.asarray(img[lv])
        h, w = im.shape
        cx = int(np.floor(px / 2 ** lv + 0.5)) - 8
        cy = int(np.floor(py / 2 ** lv + 0.5)) - 8
        for r in range(16):
            for c in range(16):
                yy, xx = cy + r, cx + c
                if 0 <= yy < h and 0 <= xx < w:
                    x[ch, r, c] = (float(im[yy, xx]) - 128.0) / 64.0
    return x
