"""Pins for the oracle's 3x3 convolution (the surrogate network's building
block): the forward pass against scipy's 2-D cross-correlation, the backward
pass against central finite differences of the forward pass."""
import numpy as np
from scipy.signal import correlate2d

from oracle import oracle as O


def test_forward_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    B, C, Oc, H, W = 2, 3, 4, 7, 5
    x = rng.standard_normal((B, C, H, W))
    wt = rng.standard_normal((Oc, C, 3, 3))
    bias = rng.standard_normal(Oc)
    y = O.conv3x3_fwd(x, wt, bias)
    ref = np.zeros_like(y)
    for b in range(B):
        for o in range(Oc):
            ref[b, o] = bias[o] + sum(correlate2d(x[b, c], wt[o, c], mode="same", boundary="fill")
                                      for c in range(C))
    assert np.abs(y - ref).max() < 1e-12


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    B, C, Oc, H, W = 1, 2, 3, 5, 4
    x = rng.standard_normal((B, C, H, W))
    wt = rng.standard_normal((Oc, C, 3, 3))
    bias = rng.standard_normal(Oc)
    gy = rng.standard_normal((B, Oc, H, W))
    gx, gw, gb = O.conv3x3_bwd(x, wt, gy)
    f = lambda x_, w_, b_: float(np.sum(gy * O.conv3x3_fwd(x_, w_, b_)))
    h = 1e-6
    for arr, g in ((x, gx), (wt, gw), (bias, gb)):
        num = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            d = np.zeros_like(arr)
            d[idx] = h
            args = [x, wt, bias]
            k = [a is arr for a in args].index(True)
            ap, am = list(args), list(args)
            ap[k] = arr + d
            am[k] = arr - d
            num[idx] = (f(*ap) - f(*am)) / (2 * h)
        assert np.abs(num - g).max() < 1e-7 * max(1.0, np.abs(g).max())


def test_zero_padding_at_borders():
    x = np.ones((1, 1, 3, 3))
    wt = np.ones((1, 1, 3, 3))
    y = O.conv3x3_fwd(x, wt)
    assert np.array_equal(y[0, 0], np.array([[4, 6, 4], [6, 9, 6], [4, 6, 4]], dtype=float))
