"""Pins for the oracle's system matrix A (paper Eq. (sistema), Sec. II-A:
a_ij = contribution of ray i to pixel j, read as the length of ray i inside
pixel j).  The oracle clips each ray against each pixel square; these tests
check it against an independently derived closed form, brute-force sampling
along the ray, axis-aligned cases and hand-worked values."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1907_01891_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "system_matrix_2x2.json")


def _chord_through_square(p, dx, dy, a):
    """Length of the line {distance |p| from a square's centre, direction
    (dx, dy)} inside an axis-aligned square of side a.  As a function of |p| it
    is a trapezoid: a plateau a/hi for |p| <= a/2 (hi - lo), then a linear ramp
    down to zero at |p| = a/2 (hi + lo), where hi/lo = max/min(|dx|, |dy|)."""
    hi = np.maximum(np.abs(dx), np.abs(dy))
    lo = np.minimum(np.abs(dx), np.abs(dy))
    ap = np.abs(p)
    plateau = 0.5 * a * (hi - lo)
    edge = 0.5 * a * (hi + lo)
    with np.errstate(divide="ignore", invalid="ignore"):
        ramp = (edge - ap) / (hi * lo)
    return np.where(ap <= plateau, a / hi, np.where(ap < edge, ramp, 0.0))


def _rays(G):
    return np.array([O.ray(G, i) for i in range(G.n_views * G.n_bins)])


@pytest.mark.parametrize("geom", [I.parallel_geometry(16, 23, 25), I.fan_geometry(12, 17, 21),
                                  I.parallel_geometry(8, 7, 13, pixel=0.37)])
def test_matches_closed_form_chord_lengths(geom):
    G = O.Geometry(*geom.as_tuple())
    A = O.system_matrix(G)
    R = _rays(G)
    px, py, dx, dy = (R[:, k][:, None] for k in range(4))
    j = np.arange(geom.n)
    cx = (-0.5 * geom.nx + (j % geom.nx) + 0.5) * geom.pixel
    cy = (-0.5 * geom.ny + (j // geom.nx) + 0.5) * geom.pixel
    p = (cx[None, :] - px) * dy - (cy[None, :] - py) * dx
    L = _chord_through_square(p, dx, dy, geom.pixel)
    lo = np.minimum(np.abs(dx), np.abs(dy))
    # the closed form's ramp has slope 1/(hi*lo); compare where it is well conditioned
    ok = np.broadcast_to(lo > 1e-6, A.shape)
    assert ok.sum() > 0.8 * A.size
    assert np.abs(A - L)[ok].max() <= 1e-11 * geom.pixel


def test_row_sums_are_chords_through_the_image():
    geom = I.fan_geometry(20, 31, 29)
    G = O.Geometry(*geom.as_tuple())
    A = O.system_matrix(G)
    R = _rays(G)
    px, py, dx, dy = R.T
    p = (0.0 - px) * dy - (0.0 - py) * dx
    chord = _chord_through_square(p, dx, dy, geom.fov)
    assert np.allclose(A.sum(axis=1), chord, rtol=0, atol=1e-10)


def test_brute_force_sampling_along_rays():
    """Walk each ray in steps of h and count the samples falling in every
    pixel: count*h approximates a_ij to within ~2h."""
    geom = I.fan_geometry(10, 5, 9)
    G = O.Geometry(*geom.as_tuple())
    A = O.system_matrix(G)
    h = 2e-4
    x0 = -0.5 * geom.fov
    for i in range(geom.m):
        px, py, dx, dy = O.ray(G, i)
        t = np.arange(-3 * geom.src_iso, 3 * geom.src_iso, h) + 0.5 * h
        x, y = px + t * dx, py + t * dy
        ix = np.floor((x - x0) / geom.pixel).astype(np.int64)
        iy = np.floor((y - x0) / geom.pixel).astype(np.int64)
        inside = (ix >= 0) & (ix < geom.nx) & (iy >= 0) & (iy < geom.ny)
        est = np.bincount(iy[inside] * geom.nx + ix[inside], minlength=geom.n) * h
        assert np.abs(est - A[i]).max() <= 3 * h


def test_axis_aligned_rays_get_whole_pixel_widths():
    # 9 bins spaced 0.9 apart: offsets s_b = (b - 4)*0.9, all strictly inside the image
    geom = I.ScanGeometry(0, 8, 8, 1.0, 2, 9, 0.0, math.pi, 0.0, 8.1)
    G = O.Geometry(*geom.as_tuple())
    A = O.system_matrix(G)
    for b in range(geom.n_bins):  # view 0: theta = 0 exactly, rays y = s_b
        s = (b - 4) * (8.1 / 9)
        row = np.zeros(geom.n)
        iy = math.floor(s + 4)
        row[iy * 8: iy * 8 + 8] = 1.0
        assert np.array_equal(A[b], row)
    for b in range(geom.n_bins):  # view 1: theta = pi/2 (cos(pi/2) is 6e-17 in FP64), rays x ~ -s_b
        i = geom.n_bins + b
        assert np.isclose(A[i].sum(), 8.0, atol=1e-13)
        assert np.all((np.abs(A[i]) < 1e-13) | (np.abs(A[i] - 1.0) < 1e-13))
        assert np.count_nonzero(A[i] > 0.5) == 8


def test_hand_worked_golden_values():
    data = json.load(open(GOLDEN))
    im = data["image"]
    for case in data["cases"]:
        gg = case["geometry"]
        G = O.Geometry(gg["beam"], im["nx"], im["ny"], im["pixel"], gg["n_views"], gg["n_bins"],
                       gg["angle0"], gg["angle_span"], gg["src_iso"], gg["det_span"])
        A = O.system_matrix(G)
        assert np.abs(A - np.array(case["A"])).max() <= case["tol"], case["derivation"]


def test_fan_rays_start_at_source_and_fan_is_symmetric():
    geom = I.fan_geometry(16, 8, 11)
    G = O.Geometry(*geom.as_tuple())
    for v in range(geom.n_views):
        beta = v * 2 * math.pi / geom.n_views
        c = O.ray(G, v * geom.n_bins + 5)  # central bin
        assert np.allclose(c[:2], [geom.src_iso * math.cos(beta), geom.src_iso * math.sin(beta)], atol=1e-12)
        assert abs(c[0] * c[3] - c[1] * c[2]) < 1e-12  # passes through the origin
        l, r = O.ray(G, v * geom.n_bins + 0), O.ray(G, v * geom.n_bins + 10)
        ang = lambda q: math.atan2(q[3], q[2])
        assert abs((ang(l) - ang(c) + math.pi) % (2 * math.pi) - math.pi + ((ang(r) - ang(c) + math.pi) % (2 * math.pi) - math.pi)) < 1e-12


def test_config_geometries_have_no_empty_columns():
    for cfg in (I.CONFIG1,):
        g = cfg["geom"]
        A = O.system_matrix(O.Geometry(*g.as_tuple()))
        assert (A.sum(axis=0) > 0).all()
        assert A.min() >= 0.0


ANGLES = os.path.join(os.path.dirname(__file__), "golden", "view_angles_eq_angulos.json")


def test_view_angles_follow_the_quarter_shifts_of_eq_angulos():
    """The oracle's angle rule 1 against hand-worked angles of Eq. (angulos)
    (tests/golden/view_angles_eq_angulos.json states the reading)."""
    spec = json.load(open(ANGLES))
    for case in spec["cases"]:
        g = I.scanner_geometry(16, case["views"], 21)
        G = O.Geometry(*g.as_tuple())
        got = [math.degrees(O.view_angle(G, i - 1)) for i in case["i"]]
        assert np.allclose(got, case["degrees"], rtol=0, atol=1e-9), (case["views"], got)
        # angle rule 0 is the uniform spacing
        G0 = O.Geometry(*I.scanner_geometry(16, case["views"], 21, angle_rule=0).as_tuple())
        assert np.allclose([math.degrees(O.view_angle(G0, i - 1)) for i in case["i"]],
                           [360.0 * (i - 1) / case["views"] for i in case["i"]], atol=1e-9)


def test_scanner_geometry_has_the_papers_scan_dimensions():
    """Table scanner: 1025 detectors x 260 projections, 512 x 512 pixels, i.e.
    a 266,500 x 262,144 system (Sec. III); the fan of 30 degrees from 75 cm
    just covers the image's circumscribed circle."""
    g = I.scanner_geometry(512, 260, 1025)
    assert (g.m, g.n) == (266500, 262144)
    assert math.isclose(math.degrees(g.det_span), 30.0)
    half_diag = g.nx * g.pixel * math.sqrt(2.0) / 2.0
    assert math.isclose(g.src_iso * math.sin(g.det_span / 2.0), half_diag, rel_tol=1e-12)


def test_row_sums_are_chords_with_shifted_views():
    """With the angle shifts every row sum is still the chord of its ray
    through the whole image square."""
    geom = I.scanner_geometry(12, 20, 17)
    G = O.Geometry(*geom.as_tuple())
    A = O.system_matrix(G)
    R = _rays(G)
    side = geom.nx * geom.pixel
    chord = _chord_through_square(R[:, 0] * R[:, 3] - R[:, 1] * R[:, 2], R[:, 2], R[:, 3], side)
    ok = np.minimum(np.abs(R[:, 2]), np.abs(R[:, 3])) > 1e-6
    assert np.abs(A.sum(axis=1) - chord)[ok].max() <= 1e-10
