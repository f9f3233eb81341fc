"""Plain FP64 CPU model of the convolutional surrogate and its gate.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library and never imports it.

The paper has no learned part; the network here is the one the library's
``ct_surrogate_*`` entry points define (its definition is restated in the
functions below).  The convolution itself is the oracle's C routine
(``oracle.conv3x3_fwd`` / ``conv3x3_bwd``), pinned against scipy and finite
differences; the composition (residual layers, ReLU, mean-squared loss, Adam,
the gate) is pinned by central finite differences and closed forms in
``tests/test_oracle_surrogate.py``.

Storage precision.  The library keeps weights and activations in BF16 and
accumulates in FP32.  With ``bf16=True`` the model rounds to BF16 (round to
nearest even, through FP32 as the library does) at exactly the points where
the library stores a BF16 value: the scaled input, the weights, every ReLU
output and every residual sum; all arithmetic between those points is FP64.
With ``bf16=False`` it is the exact FP64 network.

Parameters are one flat FP32/FP64 vector: for each layer its weights
``[out][in][3][3]`` followed by its ``out`` biases, layers in order.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def layer_shapes(channels: int = 32, layers: int = 6):
    """[(cin, cout)] of the network: 1 -> C, (L - 2) x (C -> C), C -> 1."""
    return [(1, channels)] + [(channels, channels)] * (layers - 2) + [(channels, 1)]


def num_params(channels: int = 32, layers: int = 6) -> int:
    return sum(co * ci * 9 + co for ci, co in layer_shapes(channels, layers))


def unpack(params, channels: int = 32, layers: int = 6):
    """[(W[out, in, 3, 3], b[out])] views of the flat parameter vector."""
    out, off = [], 0
    for ci, co in layer_shapes(channels, layers):
        w = np.asarray(params[off:off + co * ci * 9], dtype=np.float64).reshape(co, ci, 3, 3)
        off += co * ci * 9
        b = np.asarray(params[off:off + co], dtype=np.float64)
        off += co
        out.append((w, b))
    assert off == len(params)
    return out


def round_bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), first to FP32."""
    f = np.atleast_1d(np.asarray(x, dtype=np.float64)).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    r = r.astype(np.uint32).view(np.float32).astype(np.float64)
    r[np.isnan(f)] = np.nan
    return r.reshape(np.shape(x))


def forward(params, g, in_scale: float, channels: int = 32, layers: int = 6, bf16: bool = True):
    """Network output y (B, 1, H, W) for backprojections g (B, H, W) and the
    cache the backward pass needs.

    a1 = relu(conv0(in_scale * g)); a_{l+1} = a_l + relu(conv_l(a_l)) for the
    middle layers; y = conv_{L-1}(a_{L-1}).
    """
    rnd = round_bf16 if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    P = unpack(params, channels, layers)
    Wb = [(rnd(w), b) for w, b in P]
    a = [rnd(np.asarray(g, dtype=np.float64)[:, None] * in_scale)]
    r = [None]
    w0, b0 = Wb[0]
    r.append(rnd(np.maximum(O.conv3x3_fwd(a[0], w0, b0), 0.0)))
    a.append(r[1])
    for l in range(1, layers - 1):
        w, b = Wb[l]
        r.append(rnd(np.maximum(O.conv3x3_fwd(a[l], w, b), 0.0)))
        a.append(rnd(a[l] + r[l + 1]))
    wl, bl = Wb[layers - 1]
    y = O.conv3x3_fwd(a[layers - 1], wl, bl)
    return y, dict(a=a, r=r, W=[w for w, _ in Wb])


def loss_and_grad(params, g, x, in_scale: float, out_scale: float, channels: int = 32, layers: int = 6,
                  bf16: bool = True):
    """Loss mean((y - x / out_scale)^2) over all pixels of all images and its
    gradient with respect to the flat parameter vector (backpropagation through
    the network of ``forward``; ReLU derivative 1 where its output is > 0)."""
    y, c = forward(params, g, in_scale, channels, layers, bf16)
    t = np.asarray(x, dtype=np.float64)[:, None] / out_scale
    d = y - t
    n = d.size
    loss = float(np.sum(d * d) / n)
    dy = 2.0 * d / n
    grads = [None] * layers
    a, r, W = c["a"], c["r"], c["W"]
    dA, gw, gb = O.conv3x3_bwd(a[layers - 1], W[layers - 1], dy)
    grads[layers - 1] = (gw, gb)
    for l in range(layers - 2, 0, -1):
        dz = np.where(r[l + 1] > 0.0, dA, 0.0)
        dx, gw, gb = O.conv3x3_bwd(a[l], W[l], dz)
        grads[l] = (gw, gb)
        dA = dA + dx
    dz = np.where(r[1] > 0.0, dA, 0.0)
    _, gw, gb = O.conv3x3_bwd(a[0], W[0], dz)
    grads[0] = (gw, gb)
    flat = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in grads])
    return loss, flat


def adam_step(p, m, v, grad, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma and Ba, 2015) with bias correction at step t >= 1;
    returns the new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def gate(A, xhat, b, tol: float):
    """Per-slice residual ||A xhat - b|| / ||b|| (||A xhat|| when b = 0) and
    whether it passes (<= tol; NaN fails).  A is m x n, xhat n x k, b m x k."""
    R = A @ xhat - b
    rn = np.sqrt(np.sum(R * R, axis=0))
    bn = np.sqrt(np.sum(b * b, axis=0))
    res = np.where(bn > 0.0, rn / np.where(bn > 0.0, bn, 1.0), rn)
    return res, res <= tol
