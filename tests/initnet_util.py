"""Shared helpers of the flow network's gradient tests (GPU and host
emulation): the per-element gradient bound and the kink margin that keeps
every ReLU decision the same on both sides."""
import numpy as np

from oracle import initnet as onet


def _kink_margin(p, x):
    """Smallest |pre-activation| / (sum of the |terms| it adds up) of one
    sample, over every ReLU input (FP64, BF16 activations)."""
    _, a = onet.forward(p, x, keep=True, act_bf16=True)
    ab = {k: np.abs(v) for k, v in p.items()}
    sums = (onet.conv_s2(np.abs(x), ab["w1"], ab["b1"]), onet.conv_s2(a["h1"], ab["w2"], ab["b2"]),
            onet.conv_s2(a["h2"], ab["w3"], ab["b3"]), ab["w4"] @ a["f"] + ab["b4"])
    pre = (a["a1"], a["a2"], a["a3"], a["a4"])
    return min(float((np.abs(u) / np.maximum(s_, 1e-300)).min()) for u, s_ in zip(pre, sums))


def _abs_grad(p, xs, flows, radius):
    """Per parameter, the mean over the batch of the sum of the |terms| that
    make up its gradient: the backward pass with every factor replaced by its
    magnitude (ReLU masks as they are)."""
    ab = {k: np.abs(v) for k, v in p.items()}
    acc = {k: np.zeros(onet.SHAPES[k]) for k in onet.ORDER}
    for x, f in zip(xs, flows):
        o, act = onet.forward(p, x, keep=True, act_bf16=True)
        _, do = onet.loss_and_grad_out(o, f, radius)
        act_abs = {k: (v if k.startswith("a") else np.abs(v)) for k, v in act.items()}
        g = onet.backward(ab, act_abs, np.abs(do))
        for k in onet.ORDER:
            acc[k] += g[k]
    return {k: v / len(xs) for k, v in acc.items()}


# Per-element gradient bound. Both sides multiply the same BF16 weights and
# BF16-stored activations; the GPU sums in FP32 (relative error ~1e-6) and can
# store an activation one BF16 step (2^-8 relative) away from the oracle's
# where the exact value sits next to a rounding tie. A gradient element is a
# sum of products with at most four such factors on its path, so it moves by
# at most 4 * 2^-8 times the sum of the |terms| it adds up (_abs_grad).
# Samples are kept only where every ReLU input lies at least 2e-5 of its
# |terms| away from zero (FP32 accumulation of up to 288 terms stays inside
# that), so no ReLU mask can differ between the two sides.
GRAD_REL = 4 * 2.0 ** -8
KINK_MARGIN = 2e-5
