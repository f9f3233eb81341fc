"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  This module holds none of the reconstruction arithmetic: it only
describes scanner geometries, draws ellipse phantoms and simulates photon noise
on projections that were computed elsewhere.

The paper reconstructs the Forbild head phantom and DeepLesion slices; neither
data set is available here, so seeded random-ellipse phantoms (piecewise
constant attenuation maps of the same kind) stand in for them.

Conventions (shared with the library and the oracle): the image has nx*ny
square pixels of side ``pixel`` centred on the origin; pixel j = iy*nx + ix,
ix along +x, iy along +y; a phantom is returned as a flat length-n vector in
that order.  Rays are numbered ray = view*n_bins + bin.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PARALLEL, FAN = 0, 1


@dataclasses.dataclass(frozen=True)
class ScanGeometry:
    """Scanner description (fields mirror ``ct_geometry`` in include/ctqr.h).

    beam PARALLEL: det_span = detector width in image units, bins centred.
    beam FAN: equiangular fan, det_span = total fan angle (radians),
              src_iso = source-to-isocentre distance.
    View v is at angle0 + v*angle_span/n_views.
    """

    beam: int
    nx: int
    ny: int
    pixel: float
    n_views: int
    n_bins: int
    angle0: float
    angle_span: float
    src_iso: float
    det_span: float
    angle_rule: int = 0   # 1: views shifted per quarter as Eq. (angulos)

    @property
    def m(self) -> int:
        return self.n_views * self.n_bins

    @property
    def n(self) -> int:
        return self.nx * self.ny

    @property
    def fov(self) -> float:
        return self.nx * self.pixel

    def as_tuple(self):
        return dataclasses.astuple(self)


def parallel_geometry(npix: int, n_views: int, n_bins: int, pixel: float = 1.0,
                      span: float = math.pi) -> ScanGeometry:
    """Parallel beam; the detector spans the image diagonal."""
    return ScanGeometry(PARALLEL, npix, npix, pixel, n_views, n_bins, 0.0, span,
                        0.0, npix * pixel * math.sqrt(2.0))


def fan_geometry(npix: int, n_views: int, n_bins: int, pixel: float = 1.0,
                 src_factor: float = 2.0) -> ScanGeometry:
    """Equiangular fan beam over a full circle; the source sits src_factor*FOV
    from the isocentre and the fan just covers the image's circumscribed circle."""
    fov = npix * pixel
    r_src = src_factor * fov
    gmax = math.asin((fov * math.sqrt(2.0) / 2.0) / r_src)
    return ScanGeometry(FAN, npix, npix, pixel, n_views, n_bins, 0.0, 2.0 * math.pi,
                        r_src, 2.0 * gmax)


def scanner_geometry(npix: int, n_views: int, n_bins: int, angle_rule: int = 1) -> ScanGeometry:
    """The paper's simulated fan-beam scanner (Table scanner): 360 degree
    circular scan, source 75 cm from the isocentre (source-to-detector 150 cm),
    30 degree fan, views at the quarter-shifted angles of Eq. (angulos).  The
    image is the square inscribed in the fan's field of view (radius
    75 sin 15 deg = 19.4 cm), so a 512 x 512 image has 0.536 mm pixels; lengths
    are in pixel units.  The paper's own scan is scanner_geometry(512, 260,
    1025): 266,500 rays x 262,144 pixels."""
    r_src_cm, half_fan = 75.0, math.radians(15.0)
    side_cm = 2.0 * r_src_cm * math.sin(half_fan) / math.sqrt(2.0)
    pixel_cm = side_cm / npix
    return ScanGeometry(FAN, npix, npix, 1.0, n_views, n_bins, 0.0, 2.0 * math.pi,
                        r_src_cm / pixel_cm, 2.0 * half_fan, angle_rule)


# The five workloads (sizes, seeds, noise) the tests and the benchmark use.
# lam > 0 stacks lam*I under the ray rows.  The 256x256 fan geometry has
# only 1.06 rays per pixel and its A is numerically rank deficient (scaled
# analogues have condition numbers near 1e17), so that workload is solved as
# the Tikhonov-stacked system [A; 1e-3 I] x = [b; 0].
CONFIG1 = dict(name="parallel32_60x45_k1", geom=parallel_geometry(32, 60, 45),
               seeds=[1], n_ellipses=5, noise_i0=None, lam=0.0)
CONFIG2 = dict(name="fan128_128x181_k16", geom=fan_geometry(128, 128, 181),
               seeds=list(range(100, 116)), n_ellipses=5, noise_i0=1e5, lam=0.0)
CONFIG3 = dict(name="fan256_192x363_k64_lam1e-3", geom=fan_geometry(256, 192, 363),
               seeds=list(range(200, 264)), n_ellipses=5, noise_i0=None, lam=1e-3)
CONFIG4A = dict(name="parallel32_60x45_k512", geom=parallel_geometry(32, 60, 45),
                seeds=list(range(1000, 1512)), n_ellipses=5, noise_i0=1e4, lam=0.0)
# 64 uneven lambda-stacked systems (geometries from uneven_systems(64, 4242)),
# one noiseless phantom each (seed 2000 + system index).
CONFIG4B = dict(name="fan_uneven32-96_x64_lam1e-3", count=64, seed=4242, seed0=2000, n_ellipses=5,
                lam=1e-3)
# Learned surrogate on the 128 x 128 fan-beam scan (noiseless b = A x):
# training phantoms 20000 seeds, inference batch 256 on unseen seeds.
CONFIG5 = dict(name="fan128_surrogate_train20000_k256", geom=fan_geometry(128, 128, 181),
               train_seeds=range(10_000, 30_000), seeds=list(range(50_000, 50_256)), n_ellipses=5,
               noise_i0=None, lam=0.0, tol=1e-3)


def uneven_systems(count: int = 64, seed: int = 4242, npix_range=(32, 96), ratio_range=(1.2, 2.0)):
    """Seeded fan-beam geometries of uneven size: image side uniform in
    npix_range, rays per pixel uniform in ratio_range (detector bins ~1.42 x the
    side, rounded to odd; views = rays / bins)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        npix = int(rng.integers(npix_range[0], npix_range[1] + 1))
        ratio = float(rng.uniform(*ratio_range))
        bins = int(math.ceil(1.42 * npix)) | 1
        views = max(2, int(round(ratio * npix * npix / bins)))
        out.append(fan_geometry(npix, views, bins))
    return out


def ellipse_phantom(nx: int, ny: int, pixel: float, seed: int, n_ellipses: int = 5) -> np.ndarray:
    """Sum of n_ellipses random ellipses sampled at pixel centres.

    Centres uniform in a disc of radius 0.3*FOV, semi-axes U[0.05, 0.4]*FOV,
    rotation U[0, pi), density U[0.1, 1]; overlapping ellipses add.
    """
    rng = np.random.default_rng(seed)
    fov = max(nx, ny) * pixel
    xs = (np.arange(nx) + 0.5) * pixel - 0.5 * nx * pixel
    ys = (np.arange(ny) + 0.5) * pixel - 0.5 * ny * pixel
    X, Y = np.meshgrid(xs, ys)  # Y[iy, ix], X[iy, ix]
    img = np.zeros((ny, nx))
    for _ in range(n_ellipses):
        r = 0.3 * fov * math.sqrt(rng.uniform())
        phi = rng.uniform(0.0, 2.0 * math.pi)
        cx, cy = r * math.cos(phi), r * math.sin(phi)
        a, b = rng.uniform(0.05, 0.4, size=2) * fov
        rot = rng.uniform(0.0, math.pi)
        rho = rng.uniform(0.1, 1.0)
        u = (X - cx) * math.cos(rot) + (Y - cy) * math.sin(rot)
        v = -(X - cx) * math.sin(rot) + (Y - cy) * math.cos(rot)
        img += rho * ((u / a) ** 2 + (v / b) ** 2 <= 1.0)
    return img.reshape(-1)


def phantoms(geom: ScanGeometry, seeds, n_ellipses: int = 5) -> np.ndarray:
    """n x len(seeds) column-major matrix of phantoms, one column per seed."""
    X = np.empty((geom.n, len(seeds)), order="F")
    for c, s in enumerate(seeds):
        X[:, c] = ellipse_phantom(geom.nx, geom.ny, geom.pixel, s, n_ellipses)
    return X


def poisson_noise(b: np.ndarray, fov: float, i0: float, seed: int) -> np.ndarray:
    """Replace exact projections b (line integrals in pixel-length units) by
    noisy ones: with p = b/fov, counts y ~ Poisson(i0*exp(-p)) and
    b_noisy = -ln(max(y, 1)/i0) * fov.  Drawn with numpy's PCG64."""
    rng = np.random.default_rng(seed)
    p = np.asarray(b, dtype=np.float64) / fov
    y = rng.poisson(i0 * np.exp(-p)).astype(np.float64)
    return np.asfortranarray(-np.log(np.maximum(y, 1.0) / i0) * fov)


def random_matrix(m: int, n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Column-major standard-normal matrix (generic parity inputs)."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((m, n)).astype(dtype))
