"""Learned warm start for the level-1 eigenproblems: the reference computation
of the network, its loss, gradients and Adam step, FP64 NumPy.

Test infrastructure only (see the package docstring).  Not a step of the
paper: the network only seeds the level-1 subspace iteration, which still runs
to the eigen-residual tolerance, so the preconditioner does not depend on it.

Parameters are one flat array with the layout of the library (weight matrix
l row-major [fan_in][fan_out] at w_off[l], bias at b_off[l]); the layout is an
input here.  The products read BF16 operands, as the library's tensor-core
products do: the weights rounded to BF16 (``bf16_round``) and the activations
x, h1, h2 rounded to BF16 before the product that reads them (after rounding
the exact value to FP32, the precision in which the library accumulates).
Gradients are taken with respect to the rounded weights, through the rounding
of the activations as through the identity, and applied to the FP32 masters.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even) and
    return them as float64: keep the top 16 bits of the float32 pattern after
    adding 0x7FFF plus the lowest kept bit (finite inputs)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params: np.ndarray, dims, w_off, b_off, round_weights: bool = True):
    """(W_l, b_l) for l = 0, 1, 2; dims = (n_in, h1, h2, n_out)."""
    p = np.asarray(params)
    Ws, bs = [], []
    for l in range(3):
        w = p[w_off[l]:w_off[l] + dims[l] * dims[l + 1]].reshape(dims[l], dims[l + 1])
        Ws.append(bf16_round(w) if round_weights else w.astype(np.float64))
        bs.append(p[b_off[l]:b_off[l] + dims[l + 1]].astype(np.float64))
    return Ws, bs


def out_weight(x: np.ndarray) -> np.ndarray:
    """w_c = sqrt(S_c / sum_c S_c) per row, from x_c = (log S_c - mean) / 8, i.e.
    S_c proportional to exp(8 x_c)."""
    x = np.asarray(x, dtype=np.float64)
    e = np.exp(8.0 * (x - x.max(axis=-1, keepdims=True)))
    return np.sqrt(e / e.sum(axis=-1, keepdims=True))


def forward(Ws, bs, x: np.ndarray, acts: bool = False):
    """h1 = relu(x' W1 + b1), h2 = relu(h1' W2 + b2), o = h2' W3 + b3, with ' the
    rounding of an activation to BF16, and the output y_k = w * o_k with
    w = out_weight(x) (the network predicts phi; y = S^{1/2} phi up to the
    element's normalisation).  Returns (h1, h2, y), or with ``acts`` also the
    rounded operands (x', h1', h2')."""
    x = np.asarray(x, dtype=np.float64)
    xr = bf16_round(x)
    h1 = np.maximum(xr @ Ws[0] + bs[0], 0.0)
    h1r = bf16_round(h1)
    h2 = np.maximum(h1r @ Ws[1] + bs[1], 0.0)
    h2r = bf16_round(h2)
    o = h2r @ Ws[2] + bs[2]
    B, n_in = x.shape
    y = (o.reshape(B, -1, n_in) * out_weight(x)[:, None, :]).reshape(B, -1)
    if acts:
        return h1, h2, y, (xr, h1r, h2r)
    return h1, h2, y


def loss_and_grad(out: np.ndarray, target: np.ndarray, n_vec: int):
    """Mean over samples and vectors of ||p||^2 + ||t||^2 - 2 |p . t| (the smaller
    of ||p - t||^2 and ||p + t||^2: eigenvectors have no sign), and its gradient
    with respect to out."""
    B = out.shape[0]
    p = np.asarray(out, dtype=np.float64).reshape(B, n_vec, -1)
    t = np.asarray(target, dtype=np.float64).reshape(B, n_vec, -1)
    pt = np.einsum("bki,bki->bk", p, t)
    per = (p * p).sum(-1) + (t * t).sum(-1) - 2.0 * np.abs(pt)
    nl = B * n_vec
    sg = np.where(pt >= 0.0, 1.0, -1.0)
    d = 2.0 * (p - sg[..., None] * t) / nl
    return per.sum() / nl, d.reshape(B, -1)


def gradients(params, dims, w_off, b_off, x, target, n_vec: int):
    """Loss and gradient (flat, parameter layout) by back-propagation."""
    Ws, bs = unpack(params, dims, w_off, b_off)
    x = np.asarray(x, dtype=np.float64)
    h1, h2, out, ops = forward(Ws, bs, x, acts=True)
    loss, dy = loss_and_grad(out, target, n_vec)
    B, n_in = x.shape
    d3 = (dy.reshape(B, -1, n_in) * out_weight(x)[:, None, :]).reshape(B, -1)
    g = np.zeros(np.asarray(params).shape, dtype=np.float64)
    pre = [None, h1, h2]                      # ReLU masks from the layer outputs
    d = d3
    for l in (2, 1, 0):
        g[w_off[l]:w_off[l] + dims[l] * dims[l + 1]] = (ops[l].T @ d).ravel()
        g[b_off[l]:b_off[l] + dims[l + 1]] = d.sum(axis=0)
        if l > 0:
            d = (d @ Ws[l].T) * (pre[l] > 0.0)
    return loss, g


def adam_step(w, g, m, v, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015) with bias correction; returns (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def features(S_elem: np.ndarray) -> np.ndarray:
    """Network input of an element from its Tr K~ values (any shape, one element
    per row): clamp(log S - mean log S, -20, 20) / 8."""
    ls = np.log(np.asarray(S_elem, dtype=np.float64))
    v = ls - ls.mean(axis=-1, keepdims=True)
    return np.clip(v, -20.0, 20.0) / 8.0
