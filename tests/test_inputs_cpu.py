"""The seeded input recipe (paper_1907_01891_gb300/inputs.py) against what the
workload table states: the uneven 64-system batch's size ranges, the ellipse
phantoms' value range and determinism, and the Poisson noise model's limits.
Host only; the inputs hold none of the method's arithmetic."""
import math

import numpy as np

from paper_1907_01891_gb300 import inputs as I


def test_uneven_batch_sizes_follow_the_recipe():
    cfg = I.CONFIG4B
    geoms = I.uneven_systems(cfg["count"], cfg["seed"])
    assert len(geoms) == 64
    for g in geoms:
        assert 32 <= g.nx <= 96 and g.nx == g.ny
        assert g.n_bins % 2 == 1 and g.n_bins == (math.ceil(1.42 * g.nx) | 1)
        rays_per_pixel = g.m / g.n
        assert 1.2 * 0.97 <= rays_per_pixel <= 2.0 * 1.03, (g.nx, rays_per_pixel)
    rows = sorted((g.m + g.n, g.n) for g in geoms)  # lambda-stacked systems
    assert rows[0] == (2387, 1024) and max(r[0] for r in rows) == 26752 and max(r[1] for r in rows) == 9216
    # the same seed gives the same batch
    again = I.uneven_systems(cfg["count"], cfg["seed"])
    assert [(g.nx, g.n_views, g.n_bins) for g in geoms] == [(g.nx, g.n_views, g.n_bins) for g in again]


def test_phantoms_are_seeded_sums_of_ellipses():
    g = I.CONFIG1["geom"]
    X = I.phantoms(g, [1, 2, 1])
    assert X.shape == (g.n, 3) and X.flags.f_contiguous
    assert np.array_equal(X[:, 0], X[:, 2]) and not np.array_equal(X[:, 0], X[:, 1])
    assert X.min() >= 0.0 and X.max() <= 5.0 and (X > 0).mean() > 0.05
    # every value is a sum of densities in [0.1, 1] of at most five ellipses
    vals = np.unique(X[:, 0])
    assert vals[0] == 0.0 and (vals[1:] >= 0.1 - 1e-15).all()


def test_poisson_noise_model_limits():
    g = I.CONFIG1["geom"]
    b = np.linspace(0.0, 3.0 * g.fov, 2000)[:, None]
    # very high dose: the noisy line integrals approach the exact ones
    hi = I.poisson_noise(b, g.fov, 1e14, seed=5)
    assert np.abs(hi - b).max() <= 1e-4 * g.fov
    # seeded, and low dose is noisier than high dose
    lo1, lo2 = I.poisson_noise(b, g.fov, 1e3, seed=5), I.poisson_noise(b, g.fov, 1e3, seed=5)
    assert np.array_equal(lo1, lo2)
    assert np.abs(lo1 - b).mean() > 10 * np.abs(I.poisson_noise(b, g.fov, 1e7, seed=5) - b).mean()
    # zero counts are clamped to one count: the largest value is fov * ln(i0)
    assert lo1.max() <= g.fov * math.log(1e3) + 1e-12
