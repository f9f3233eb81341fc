"""Pins for the oracle's surrogate model (oracle/surrogate.py): the backward
pass against central finite differences of the FP64 network, the network
against closed forms (identity residual layers, positive homogeneity), the
BF16 rounding against torch's conversion and hand-worked ties, Adam's first
step against its closed form, and the gate against exact residuals."""
import numpy as np
import pytest
import torch
from scipy.signal import correlate2d

from oracle import surrogate as S


def _params(rng, channels, layers, scale=0.5):
    return rng.standard_normal(S.num_params(channels, layers)) * scale


def test_layer_layout_counts():
    assert S.num_params(32, 6) == (9 * 32 + 32) + 4 * (32 * 32 * 9 + 32) + (32 * 9 + 1)
    P = S.unpack(np.arange(S.num_params(3, 4), dtype=float), 3, 4)
    assert [w.shape for w, _ in P] == [(3, 1, 3, 3), (3, 3, 3, 3), (3, 3, 3, 3), (1, 3, 3, 3)]
    # weights of layer 0 first, then its biases, then layer 1 ...
    assert P[0][1][0] == 27 and P[1][0].ravel()[0] == 30


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    C, L, B, H, W = 3, 4, 2, 5, 6
    p = _params(rng, C, L)
    p[S.num_params(C, L) - 1] = 0.3
    g = rng.standard_normal((B, H, W))
    x = rng.standard_normal((B, H, W))
    loss, grad = S.loss_and_grad(p, g, x, 0.7, 1.3, C, L, bf16=False)
    h = 1e-6
    num = np.zeros_like(p)
    for i in range(p.size):
        d = np.zeros_like(p)
        d[i] = h
        lp, _ = S.loss_and_grad(p + d, g, x, 0.7, 1.3, C, L, bf16=False)
        lm, _ = S.loss_and_grad(p - d, g, x, 0.7, 1.3, C, L, bf16=False)
        num[i] = (lp - lm) / (2 * h)
    assert np.abs(num - grad).max() <= 1e-6 * max(1.0, np.abs(grad).max())
    assert loss > 0


def test_residual_layers_with_zero_weights_are_identity():
    # Middle layers with zero weights and biases add relu(0) = 0: the network
    # reduces to conv_last(relu(conv_0(g'))), written here with scipy.
    rng = np.random.default_rng(4)
    C, L, B, H, W = 2, 5, 1, 6, 7
    p = _params(rng, C, L)
    P = S.unpack(p, C, L)
    off = 0
    for l, (w, b) in enumerate(P):
        n = w.size + b.size
        if 0 < l < L - 1:
            p[off:off + n] = 0.0
        off += n
    P = S.unpack(p, C, L)
    g = rng.standard_normal((B, H, W))
    y, _ = S.forward(p, g, 2.0, C, L, bf16=False)
    w0, b0 = P[0]
    wl, bl = P[-1]
    a1 = np.stack([np.maximum(correlate2d(2.0 * g[0], w0[c, 0], mode="same") + b0[c], 0.0) for c in range(C)])
    ref = bl[0] + sum(correlate2d(a1[c], wl[0, c], mode="same") for c in range(C))
    assert np.abs(y[0, 0] - ref).max() < 1e-12


def test_network_without_biases_is_positively_homogeneous():
    rng = np.random.default_rng(5)
    C, L = 3, 6
    p = _params(rng, C, L)
    off = 0
    for ci, co in S.layer_shapes(C, L):
        off += co * ci * 9
        p[off:off + co] = 0.0
        off += co
    g = rng.standard_normal((2, 8, 9))
    y1, _ = S.forward(p, g, 1.0, C, L, bf16=False)
    y2, _ = S.forward(p, 3.5 * g, 1.0, C, L, bf16=False)
    assert np.abs(y2 - 3.5 * y1).max() <= 1e-12 * max(1.0, np.abs(y2).max())


def test_round_bf16_ties_and_torch():
    one = 1.0
    # BF16 has 8 significant bits: neighbours of 1 are 1 +- k 2^-7 (above 1)
    assert S.round_bf16(one + 2.0 ** -8) == 1.0  # tie -> even (1.0)
    assert S.round_bf16(one + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie -> even (k = 2)
    assert S.round_bf16(one + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert np.isnan(S.round_bf16(np.array([np.nan]))[0])
    rng = np.random.default_rng(6)
    v = rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000)
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.round_bf16(v), ref)


def test_adam_first_step_closed_form():
    # After one step m_hat = g and v_hat = g^2, so p moves by -lr g / (|g| + eps).
    rng = np.random.default_rng(7)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    p1, m, v = S.adam_step(p, np.zeros(50), np.zeros(50), g, 1, 0.01)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_gate_residuals():
    rng = np.random.default_rng(8)
    A = rng.random((12, 5))
    x = rng.random((5, 4))
    b = A @ x
    xh = x.copy()
    xh[:, 1] *= 1.0 + 1e-4  # residual exactly 1e-4 of ||b||
    xh[:, 2] *= 1.0 + 1e-2
    xh[:, 3] = np.nan
    res, ok = S.gate(A, xh, b, 1e-3)
    assert res[0] < 1e-15 and abs(res[1] - 1e-4) < 1e-12 and abs(res[2] - 1e-2) < 1e-10
    assert list(ok) == [True, True, False, False]
    res0, ok0 = S.gate(A, np.zeros((5, 1)), np.zeros((12, 1)), 1e-3)
    assert res0[0] == 0.0 and ok0[0]


@pytest.mark.parametrize("bf16", [False, True])
def test_bf16_model_close_to_fp64_model(bf16):
    # The BF16-storage model stays within a few BF16 ulps (relative) of the
    # exact FP64 network on a small random case.
    rng = np.random.default_rng(9)
    C, L = 4, 6
    p = _params(rng, C, L, 0.3)
    g = rng.standard_normal((1, 8, 8))
    y64, _ = S.forward(p, g, 1.0, C, L, bf16=False)
    y, _ = S.forward(p, g, 1.0, C, L, bf16=bf16)
    err = np.linalg.norm(y - y64) / np.linalg.norm(y64)
    assert err < (5e-2 if bf16 else 1e-15)
