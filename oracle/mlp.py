"""FP64 reference of the surrogate network (test infrastructure only).

Network: 5 -> 128 -> 128 -> 128 -> 2, tanh on the hidden layers, linear
output; loss L = (1 / 2B) sum over the batch and both outputs of (y - t)^2.
Parameters follow the usual row convention: layer l maps x (B x in) to
x W_l^T + b_l with W_l of shape (out, in).

The surrogate is specified with BF16 weights and FP32 accumulation.  With
``bf16=True`` every matrix-product operand (weights, layer inputs, output
gradients) is rounded to BF16 (round to nearest even) exactly where the CUDA
kernels round it, and the products are then taken in FP64; with ``bf16=False``
everything is FP64 (used by the finite-difference pin).

Parity status: forward, backward and Adam are pinned (finite differences,
closed-form first Adam step).
"""
from __future__ import annotations

import numpy as np

SIZES = (5, 128, 128, 128, 2)


def round_bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = (bits + 0x7FFF + lsb) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def _op(a, bf16):
    return round_bf16(a) if bf16 else np.asarray(a, dtype=np.float64)


def forward(params, X, bf16=True):
    """params: list of (W, b); returns outputs and the cache for backward."""
    acts = [np.asarray(X, dtype=np.float64)]
    pre = []
    h = acts[0]
    for li, (W, b) in enumerate(params):
        z = _op(h, bf16) @ _op(W, bf16).T + b
        pre.append(z)
        h = np.tanh(z) if li < len(params) - 1 else z
        acts.append(h)
    return h, (acts, pre)


def loss(Y, T):
    return 0.5 * np.sum((Y - T) ** 2) / Y.shape[0]


def backward(params, cache, Y, T, bf16=True):
    """Gradients of the loss with respect to every (W, b)."""
    acts, pre = cache
    B = Y.shape[0]
    dz = (Y - T) / B
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        gW = _op(dz, bf16).T @ _op(acts[li], bf16)
        gb = dz.sum(axis=0)
        grads[li] = (gW, gb)
        if li > 0:
            dh = _op(dz, bf16) @ _op(W, bf16)
            dz = dh * (1.0 - acts[li] ** 2)
    return grads


def adam(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba 2015, Algorithm 1); state = (m, v, t)."""
    m, v, t = state
    t += 1
    out, m2, v2 = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        new = []
        ms, vs = [], []
        for p, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = beta1 * mm + (1 - beta1) * g
            vv = beta2 * vv + (1 - beta2) * g * g
            mhat = mm / (1 - beta1 ** t)
            vhat = vv / (1 - beta2 ** t)
            new.append(p - lr * mhat / (np.sqrt(vhat) + eps))
            ms.append(mm)
            vs.append(vv)
        out.append(tuple(new))
        m2.append(tuple(ms))
        v2.append(tuple(vs))
    return out, (m2, v2, t)


def adam_state(params):
    z = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    return (z, [(a.copy(), c.copy()) for a, c in z], 0)
