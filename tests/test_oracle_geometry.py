"""Pins of the oracle's cut-cell geometry (Sec. 2.1, Fig. 1: volume
fraction, face apertures and interface segment of a cut cell) against
closed forms computed independently."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs


def halfplane_area(a, b, c):
    """Area of {(x, y) in [0,1]^2 : a x + b y + c >= 0} by adaptive
    quadrature of the covered length of each vertical line."""
    def length(x):
        r = a * x + c
        if b == 0.0:
            return 1.0 if r >= 0.0 else 0.0
        y0 = -r / b
        if b > 0:
            return min(max(1.0 - y0, 0.0), 1.0)
        return min(max(y0, 0.0), 1.0)
    pts = []
    if a != 0.0:
        for yy in (0.0, 1.0):
            xx = -(b * yy + c) / a
            if 0.0 < xx < 1.0:
                pts.append(xx)
    val, _ = quad(length, 0.0, 1.0, points=sorted(pts) or None, epsabs=1e-15, epsrel=1e-14, limit=200)
    return val


def test_edge_fraction_linear_crossing():
    assert O.edge_fraction(1.0, 2.0) == 1.0
    assert O.edge_fraction(-1.0, -2.0) == 0.0
    assert O.edge_fraction(0.0, -1.0) == 0.0 or O.edge_fraction(0.0, -1.0) == 0.0
    assert O.edge_fraction(1.0, -3.0) == pytest.approx(0.25, abs=1e-16)
    assert O.edge_fraction(-3.0, 1.0) == pytest.approx(0.25, abs=1e-16)
    assert O.edge_fraction(-1.0, 1.0) == pytest.approx(0.5, abs=1e-16)


@pytest.mark.parametrize("seed", range(40))
def test_cell_alpha_equals_exact_halfplane_area(seed):
    rng = np.random.default_rng(seed)
    th = rng.uniform(0, 2 * np.pi)
    a, b = math.cos(th), math.sin(th)
    c = rng.uniform(-1.2, 0.6)
    f = lambda x, y: a * x + b * y + c
    got = O.cell_alpha(f(0, 0), f(1, 0), f(1, 1), f(0, 1))
    assert got == pytest.approx(halfplane_area(a, b, c), abs=1e-12)


def test_saddle_takes_disconnected_corner_triangles():
    # P at (0,0) and (1,1); crossings at edge midpoints: two triangles 1/8
    assert O.cell_alpha(1.0, -1.0, 1.0, -1.0) == pytest.approx(0.25, abs=1e-15)
    assert O.cell_alpha(-1.0, 1.0, -1.0, 1.0) == pytest.approx(0.25, abs=1e-15)


def _plane_case(angle, off, n=16):
    d = 1.0 / n
    mat = {"gamma": 1.4, "pinf": 0.0}
    cfg = inputs.config(n, n, d, d, mat, mat, ["zerograd"] * 4, band=1e9)
    X, Y = inputs._centres(cfg)
    nx, ny = math.cos(angle), math.sin(angle)
    phi = (X - 0.5) * nx + (Y - 0.5) * ny - off
    pr = inputs._uniform(X.shape, 1.0, 0.0, 0.0, 1.0)
    return cfg, phi, pr, (nx, ny, off)


@pytest.mark.parametrize("angle", [0.0, 0.37, 1.1, 2.5, -0.8])
def test_plane_geometry_is_exact(angle):
    cfg, phi, pr, (nx, ny, off) = _plane_case(angle, 0.031)
    o = O.Oracle(cfg).init(phi, pr, pr)
    g = o.geometry()
    n, d = cfg["nx"], cfg["dx"]
    for j in range(2, n - 2):
        for i in range(2, n - 2):
            # cell [i d, (i+1) d] x [j d, (j+1) d] in unit coordinates
            a, b = nx * d, ny * d
            c = (i * d - 0.5) * nx + (j * d - 0.5) * ny - off
            assert g["alpha"][j, i] == pytest.approx(halfplane_area(a, b, c), abs=1e-12)
            # P length of the left face x = i d, y in [j d, (j+1) d]
            ya, yb = c, c + b
            exact_ax = 1.0 if min(ya, yb) >= 0 else (0.0 if max(ya, yb) < 0 else max(ya, yb) / abs(yb - ya))
            assert g["ax"][j, i] == pytest.approx(exact_ax, abs=1e-12)
            # interface segment: |S| equals the chord length of the line in the cell
            if 0.0 < g["alpha"][j, i] < 1.0:
                S = math.hypot(g["sx"][j, i], g["sy"][j, i])
                # chord via the area derivative: d(area)/dc = chord / |grad| in unit cell
                h = 1e-6
                chord = (halfplane_area(a, b, c + h) - halfplane_area(a, b, c - h)) / (2 * h) * math.hypot(a, b) * d
                assert S == pytest.approx(chord, rel=1e-6, abs=1e-12)
                # S points from N to P along the plane normal
                assert g["sx"][j, i] * nx + g["sy"][j, i] * ny > 0


def test_circle_area_converges_second_order():
    errs = []
    for n in (32, 64, 128):
        d = 1.0 / n
        mat = {"gamma": 1.4, "pinf": 0.0}
        cfg = inputs.config(n, n, d, d, mat, mat, ["zerograd"] * 4, band=1e9)
        X, Y = inputs._centres(cfg)
        R = 0.3
        phi = R - np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2)  # P inside
        pr = inputs._uniform(X.shape, 1.0, 0.0, 0.0, 1.0)
        o = O.Oracle(cfg).init(phi, pr, pr)
        area = o.geometry()["alpha"].sum() * d * d
        errs.append(abs(area - math.pi * R * R))
    assert errs[1] < errs[0] / 3.0 and errs[2] < errs[1] / 3.0
    assert errs[2] < 1e-4


def test_interface_vector_closes_each_cell():
    cfg, phi, pr, _ = _plane_case(0.7, 0.0)
    o = O.Oracle(cfg).init(phi, pr, pr)
    g = o.geometry()
    d = cfg["dx"]
    sx = (g["ax"][:, 1:] - g["ax"][:, :-1]) * d
    sy = (g["ay"][1:, :] - g["ay"][:-1, :]) * d
    assert np.abs(sx - g["sx"]).max() == 0.0 and np.abs(sy - g["sy"]).max() == 0.0
