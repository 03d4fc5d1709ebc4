"""ORACLE (test infrastructure only): the learned page prefetcher in FP64.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package; it shares no code with the CUDA library.

The paper has no learned component; its limitations section asks for copy
prioritisation and asynchronous transfers (Sec. 4.3 "Limitations").  The
prefetcher is the network of the scene's learned-prefetch configuration:
inputs = camera position (3), forward (3), velocity (3), angular velocity (3)
and a 256-bin histogram of the previous frame's required pages; two ReLU
hidden layers of 256; one logit per page of a 4096-page neighbourhood;
binary cross-entropy with logits averaged over the unmasked outputs; Adam.
The oracle runs on the bf16-rounded weights and inputs the GPU sees, with
FP64 arithmetic everywhere else.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a):
    """Round float values to the nearest bf16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(W, x):
    """W = dict(W1[in,h], b1[h], W2[h,h], b2[h], W3[h,out], b3[out]); x[B,in]."""
    z1 = x @ W["W1"] + W["b1"]
    h1 = np.maximum(z1, 0)
    z2 = h1 @ W["W2"] + W["b2"]
    h2 = np.maximum(z2, 0)
    y = h2 @ W["W3"] + W["b3"]
    return dict(z1=z1, h1=h1, z2=z2, h2=h2, logits=y)


def bce_with_logits(logits, target, mask):
    """mean over mask of max(x,0) - x*t + log(1 + exp(-|x|))."""
    l = np.maximum(logits, 0) - logits * target + np.log1p(np.exp(-np.abs(logits)))
    return float((l * mask).sum() / max(mask.sum(), 1))


def loss_and_grads(W, x, target, mask):
    f = forward(W, x)
    n = max(mask.sum(), 1)
    loss = bce_with_logits(f["logits"], target, mask)
    sig = 1.0 / (1.0 + np.exp(-f["logits"]))
    dy = (sig - target) * mask / n
    g = {}
    g["W3"] = f["h2"].T @ dy
    g["b3"] = dy.sum(0)
    dh2 = dy @ W["W3"].T
    dz2 = dh2 * (f["z2"] > 0)
    g["W2"] = f["h1"].T @ dz2
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ W["W2"].T
    dz1 = dh1 * (f["z1"] > 0)
    g["W1"] = x.T @ dz1
    g["b1"] = dz1.sum(0)
    return loss, g, f


def adam(W, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba), bias-corrected, t >= 1."""
    out_W, out_m, out_v = {}, {}, {}
    for k in W:
        out_m[k] = b1 * m[k] + (1 - b1) * g[k]
        out_v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = out_m[k] / (1 - b1 ** t)
        vh = out_v[k] / (1 - b2 ** t)
        out_W[k] = W[k] - lr * mh / (np.sqrt(vh) + eps)
    return out_W, out_m, out_v
