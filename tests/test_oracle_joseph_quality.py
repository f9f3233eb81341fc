"""Pins for the oracle's Joseph projector (the paper's sinogram simulator,
Sec. III) and its image-quality measures (Sec. II-D: Eq. MSE, Eq. psnr,
Eq. ssim), each against values fixed by geometry or a closed form."""
import math

import numpy as np
import pytest
from scipy import ndimage

from oracle import oracle as O
from paper_1907_01891_gb300 import inputs as I


def _G(g):
    return O.Geometry(*g.as_tuple())


def test_axis_parallel_rays_through_pixel_centres_sum_columns():
    """Vertical rays through the centres of the pixel columns (parallel beam
    at 90 degrees, one bin per column): every row contributes exactly its
    pixel, times the step p / |dy| = p."""
    nx, p = 7, 0.6
    g = I.ScanGeometry(0, nx, 5, p, 1, nx, math.pi / 2, math.pi, 0.0, nx * p)
    X = np.random.default_rng(1).uniform(0, 1, (5 * nx, 3))
    B = O.joseph_project(_G(g), X)
    img = X.reshape(5, nx, 3)                        # [iy, ix, c]
    cols = p * img.sum(axis=0)                       # [ix, c]
    # bin b's ray passes through x = ((nx-1)/2 - b) p: column nx - 1 - b
    assert np.allclose(B, cols[::-1], rtol=0, atol=1e-12)


def test_linear_image_gives_the_exact_line_integral_on_interior_rays():
    """f(x, y) = a + b x + c y sampled at the pixel centres: inside a row the
    linear interpolation is exact, and each row band's contribution is the
    midpoint rule of a linear function, also exact.  For rays that cross the
    top and bottom edges away from the side borders the projection is the
    line integral L f(x(0), 0), L = ny p / |dy|."""
    g = I.ScanGeometry(0, 24, 24, 1.0, 40, 9, 0.0, math.pi, 0.0, 8.0)
    G = _G(g)
    a, b, c = 0.7, 0.031, -0.017
    xs = (np.arange(24) + 0.5) - 12.0
    X = (a + b * xs[None, :] + c * xs[:, None]).reshape(-1)
    B = O.joseph_project(G, X)
    checked = 0
    for i in range(g.m):
        px, py, dx, dy = O.ray(G, i)
        if abs(dy) < abs(dx):
            continue
        t = np.array([(-12.0 - py) / dy, (12.0 - py) / dy])
        x_end = px + t * dx
        if np.any(np.abs(x_end) > 12.0 - 0.5 - 1e-9):   # interpolation would meet the border
            continue
        x_mid = px + (0.0 - py) / dy * dx
        L = 24.0 / abs(dy)
        assert B[i] == pytest.approx(L * (a + b * x_mid), rel=1e-12, abs=1e-12)
        checked += 1
    assert checked >= 50


def test_hand_worked_two_by_two():
    """Image [[1, 2], [3, 4]] (pixel iy*2 + ix, unit pixels, image [-1,1]^2).
    A ray at 45 degrees through the origin (|dx| = |dy|: rows): row 0 at
    y = -1/2 meets x = -1/2, the centre of pixel (0, 0); row 1 at y = 1/2
    meets x = 1/2, the centre of pixel (1, 1); step sqrt(2): (1 + 4) sqrt(2).
    A horizontal ray at y = 1/2 (columns): both columns meet row 1's centre
    line: 3 + 4 = 7."""
    X = np.array([1.0, 2.0, 3.0, 4.0])
    g45 = I.ScanGeometry(0, 2, 2, 1.0, 1, 1, math.pi / 4, math.pi, 0.0, 2.0)
    assert O.joseph_project(_G(g45), X)[0] == pytest.approx(5.0 * math.sqrt(2.0), rel=1e-14)
    gh = I.ScanGeometry(0, 2, 2, 1.0, 1, 2, 0.0, math.pi, 0.0, 2.0)   # rays at y = -1/2 and +1/2
    assert np.allclose(O.joseph_project(_G(gh), X), [1.0 + 2.0, 3.0 + 4.0], rtol=0, atol=1e-14)


def test_linear_in_the_image_and_close_to_siddon_on_smooth_images():
    g = I.fan_geometry(48, 60, 69)
    G = _G(g)
    rng = np.random.default_rng(2)
    X1, X2 = rng.uniform(0, 1, (g.n, 2)).T
    B = O.joseph_project(G, np.stack([X1, X2, 2 * X1 - 3 * X2], axis=1))
    assert np.allclose(B[:, 2], 2 * B[:, 0] - 3 * B[:, 1], rtol=1e-12, atol=1e-12)
    # a smooth blob: both projectors approximate its line integrals
    xs = (np.arange(48) + 0.5) - 24.0
    blob = np.exp(-(xs[None, :] ** 2 + xs[:, None] ** 2) / (2 * 9.0 ** 2)).reshape(-1)
    Bj = O.joseph_project(G, blob)
    Bs = O.system_matrix(G) @ blob
    assert np.linalg.norm(Bj - Bs) <= 5e-3 * np.linalg.norm(Bs)


def test_quality_of_identical_and_shifted_images():
    rng = np.random.default_rng(3)
    ref = rng.uniform(0.0, 2.0, (32 * 40))
    mse, psnr, ssim = O.quality(ref, ref, 40, 32)
    assert mse == 0.0 and math.isinf(psnr) and ssim == pytest.approx(1.0, abs=1e-12)
    d = 0.01
    mse, psnr, _ = O.quality(ref + d, ref, 40, 32)
    assert mse == pytest.approx(d * d, rel=1e-9)
    assert psnr == pytest.approx(10 * math.log10(ref.max() ** 2 / d ** 2), rel=1e-9)


def test_ssim_against_a_library_gaussian_filter():
    """The same SSIM reading computed with scipy's Gaussian filter (11 x 11
    window: sigma 1.5 truncated at radius 5, normalised) over the pixels whose
    window lies inside the image."""
    rng = np.random.default_rng(4)
    ny, nx = 30, 37
    ref = ndimage.gaussian_filter(rng.uniform(0, 1, (ny, nx)), 2.0)
    x = ref + 0.05 * rng.standard_normal((ny, nx))
    L = ref.max() - ref.min()
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    f = lambda z: ndimage.gaussian_filter(z, 1.5, truncate=5 / 1.5, mode="constant")[5:-5, 5:-5]
    mx, my = f(x), f(ref)
    vx, vy, cxy = f(x * x) - mx * mx, f(ref * ref) - my * my, f(x * ref) - mx * my
    s = ((2 * mx * my + c1) * (2 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2))
    assert O.quality(x.reshape(-1), ref.reshape(-1), nx, ny)[2] == pytest.approx(s.mean(), rel=1e-10)
