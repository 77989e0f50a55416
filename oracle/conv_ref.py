"""FP64 CPU reference of the learned super-stepper's network (test
infrastructure only; imported by ``tests/`` alone).

Plain numpy definitions of the operations the CUDA network kernels compute,
written from the textbook definitions with no blocking, fusion or
reordering:

* circular, dilated 3x3 cross-correlation on NHWC tensors,
  y[b, i, j, co] = bias[co] + sum_{ky, kx, ci} x[b, i + (ky-1) d, j + (kx-1) d, ci] w[co, 3 ky + kx, ci]
  (indices mod H and W);
* its gradients with respect to the input, the weights and the bias;
* the five-layer network (ReLU after layers 1-4 or no activation at all,
  none after layer 5) and its backward pass, the channel-weighted squared-error loss, and
* the bias-corrected Adam update (Kingma and Ba, 2015, Algorithm 1).

It shares nothing with the CUDA library.  These functions are pinned in
``tests/test_oracle_conv.py`` against scipy's circular correlation, brute
force loops and central finite differences.
"""
from __future__ import annotations

import numpy as np


def shifted(x: np.ndarray, tap: int, dil: int) -> np.ndarray:
    """xs[b, i, j] = x[b, i + (ky-1) dil, j + (kx-1) dil] (periodic), tap = 3 ky + kx."""
    ky, kx = divmod(tap, 3)
    return np.roll(x, shift=(-(ky - 1) * dil, -(kx - 1) * dil), axis=(1, 2))


def conv3x3(x, w, bias, dil):
    """x [B,H,W,Cin], w [Cout,9,Cin], bias [Cout] or None -> y [B,H,W,Cout]."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    y = np.zeros(x.shape[:3] + (w.shape[0],))
    for tap in range(9):
        y += shifted(x, tap, dil) @ w[:, tap, :].T
    if bias is not None:
        y += np.asarray(bias, dtype=np.float64)
    return y


def conv3x3_backward(x, w, dy, dil):
    """Gradients of sum(dy * conv3x3(x, w, b, dil)): returns (dx, dw, db)."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for tap in range(9):
        ky, kx = divmod(tap, 3)
        # x[q] feeds y[q - off] through tap: dx[q] += dy[q - off] w_tap
        dx += np.roll(dy @ w[:, tap, :], shift=((ky - 1) * dil, (kx - 1) * dil), axis=(1, 2))
        dw[:, tap, :] = np.einsum("bhwo,bhwi->oi", dy, shifted(x, tap, dil))
    db = dy.sum(axis=(0, 1, 2))
    return dx, dw, db


def net_forward(x, params, dils, relu=True):
    """params: list of (w, b) per layer; returns the list of layer outputs
    [a1, ..., a_L] (ReLU applied to all but the last when relu is set)."""
    acts = []
    a = np.asarray(x, dtype=np.float64)
    for li, ((w, b), d) in enumerate(zip(params, dils)):
        z = conv3x3(a, w, b, d)
        a = np.maximum(z, 0.0) if (relu and li + 1 < len(params)) else z
        acts.append(a)
    return acts


def weighted_mse(y, t, wch, scale):
    """loss = scale * sum wch[c] (y - t)^2 and its gradient with respect to y."""
    e = np.asarray(y, dtype=np.float64) - np.asarray(t, dtype=np.float64)
    wch = np.asarray(wch, dtype=np.float64)
    return scale * float(np.sum(wch * e * e)), 2.0 * scale * wch * e


def net_backward(x, params, dils, acts, dy_out, relu=True):
    """Gradients of sum(dy_out * a_L) with respect to every (w, b)."""
    grads = [None] * len(params)
    dy = np.asarray(dy_out, dtype=np.float64)
    for li in range(len(params) - 1, -1, -1):
        inp = x if li == 0 else acts[li - 1]
        dx, dw, db = conv3x3_backward(inp, params[li][0], dy, dils[li])
        grads[li] = (dw, db)
        if li > 0:
            dy = dx * (acts[li - 1] > 0) if relu else dx  # ReLU derivative of the previous layer
    return grads


def adam_step(p, g, m, v, lr, beta1, beta2, eps, t):
    """One Adam update at step t >= 1; returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
