"""Pins of the oracle's single-fluid finite-volume scheme (Sec. 4: WENO5
with Lax-Friedrichs splitting, TVD-RK2) and of its reduction from the
cut-cell update (Eq. 2) when one fluid fills the domain."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs


def test_weno5_reproduces_constants_and_linears():
    for v in ([3.0] * 5, [1.0, 2.0, 3.0, 4.0, 5.0], [-2.0, -1.5, -1.0, -0.5, 0.0]):
        got = O.weno5(v)
        # point values of a linear function: face value is v3 + (v4 - v3)/2
        assert got == pytest.approx(v[2] + 0.5 * (v[3] - v[2]), abs=1e-14)


def test_weno5_is_odd_and_essentially_non_oscillatory():
    v = np.array([1.0, 1.0, 1.0, 0.0, 0.0])
    assert O.weno5(-v) == -O.weno5(v)
    got = O.weno5(v)
    assert -1e-6 <= got <= 1.0 + 1e-6


def _smooth_single_fluid(n):
    d = 1.0 / n
    mat = {"gamma": 1.4, "pinf": 0.0}
    cfg = inputs.config(n, n, d, d, mat, mat, ["periodic"] * 4)
    X, Y = inputs._centres(cfg)
    phi = np.ones_like(X)
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    u = 0.3 + 0.1 * np.cos(2 * np.pi * Y)
    v = -0.2 + 0.1 * np.sin(2 * np.pi * X)
    p = 1.0 + 0.1 * np.cos(2 * np.pi * (X + Y))
    pr = np.stack([rho, u, v, p])
    return cfg, X, Y, phi, pr


def _exact_divergence(X, Y):
    """-div F of the smooth field, differentiated analytically."""
    s, c, tp = np.sin, np.cos, 2 * np.pi
    rho = 1.0 + 0.2 * s(tp * X) * c(tp * Y)
    rx = 0.2 * tp * c(tp * X) * c(tp * Y)
    ry = -0.2 * tp * s(tp * X) * s(tp * Y)
    u = 0.3 + 0.1 * c(tp * Y)
    uy = -0.1 * tp * s(tp * Y)
    v = -0.2 + 0.1 * s(tp * X)
    vx = 0.1 * tp * c(tp * X)
    p = 1.0 + 0.1 * c(tp * (X + Y))
    px = py = -0.1 * tp * s(tp * (X + Y))
    g = 1.4
    E = p / (g - 1) + 0.5 * rho * (u * u + v * v)
    Ex = px / (g - 1) + 0.5 * rx * (u * u + v * v) + rho * (v * vx)
    Ey = py / (g - 1) + 0.5 * ry * (u * u + v * v) + rho * (u * uy)
    # F = (rho u, rho u^2 + p, rho u v, u(E + p)); u depends on y only, v on x only
    dF0 = rx * u
    dG0 = ry * v + rho * 0.0
    dF1 = rx * u * u + px
    dG1 = ry * u * v + rho * uy * v
    dF2 = rx * u * v + rho * u * vx
    dG2 = ry * v * v + py
    dF3 = u * (Ex + px)
    dG3 = v * (Ey + py)
    return -np.stack([dF0 + dG0, dF1 + dG1, dF2 + dG2, dF3 + dG3])


def test_single_fluid_operator_is_fifth_order():
    errs = []
    for n in (16, 32, 64):
        cfg, X, Y, phi, pr = _smooth_single_fluid(n)
        o = O.Oracle(cfg).init(phi, pr, pr)
        L = o.rhs(1)
        errs.append(np.abs(L - _exact_divergence(X, Y)).max())
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 4.5, (errs, orders)


def _plain_rhs(U, lf, dx, g):
    """Standard WENO5-LF finite-volume divergence on a periodic grid, written
    without any cut-cell machinery (global Lax-Friedrichs splitting)."""
    def recon(v1, v2, v3, v4, v5, eps=1e-6):
        q0 = (2 * v1 - 7 * v2 + 11 * v3) / 6
        q1 = (-v2 + 5 * v3 + 2 * v4) / 6
        q2 = (2 * v3 + 5 * v4 - v5) / 6
        b0 = 13 / 12 * (v1 - 2 * v2 + v3) ** 2 + 0.25 * (v1 - 4 * v2 + 3 * v3) ** 2
        b1 = 13 / 12 * (v2 - 2 * v3 + v4) ** 2 + 0.25 * (v2 - v4) ** 2
        b2 = 13 / 12 * (v3 - 2 * v4 + v5) ** 2 + 0.25 * (3 * v3 - 4 * v4 + v5) ** 2
        a0, a1, a2 = 0.1 / (eps + b0) ** 2, 0.6 / (eps + b1) ** 2, 0.3 / (eps + b2) ** 2
        return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2)

    rho, mx, my, E = U
    u, v = mx / rho, my / rho
    p = (g - 1) * (E - 0.5 * rho * (u * u + v * v))
    out = np.zeros_like(U)
    for axis, vel, a in ((1, u, lf[0]), (0, v, lf[1])):
        F = np.stack([rho * vel, mx * vel + (p if axis == 1 else 0), my * vel + (p if axis == 0 else 0), vel * (E + p)])
        fp, fm = 0.5 * (F + a * U), 0.5 * (F - a * U)
        sh = lambda A, k: np.roll(A, -k, axis=axis + 1)
        # flux at the face between cells i and i+1
        Fh = recon(sh(fp, -2), sh(fp, -1), fp, sh(fp, 1), sh(fp, 2)) + \
            recon(sh(fm, 3), sh(fm, 2), sh(fm, 1), fm, sh(fm, -1))
        out += -(Fh - sh(Fh, -1)) / dx
    return out


def test_cut_cell_update_reduces_to_plain_scheme():
    cfg, X, Y, phi, pr = _smooth_single_fluid(24)
    o = O.Oracle(cfg).init(phi, pr, pr)
    L = o.rhs(1)
    qN, qP, _ = o.state()
    rho, u, v, p = pr
    c = np.sqrt(1.4 * p / rho)
    lf = (np.max(np.abs(u) + c), np.max(np.abs(v) + c))
    Lp = _plain_rhs(qP, lf, cfg["dx"], 1.4)
    scale = np.abs(Lp).max(axis=(1, 2))[:, None, None]
    assert np.abs(L - Lp).max() <= 1e-12 * scale.max()
    assert np.all(qN == 0.0)
    # and the update: a full RK2 step with alpha = 1 everywhere
    info = o.step_single_dt(1)
    assert info["err"] == 0


def test_smooth_advection_time_step_converges():
    """Density wave advected by a uniform flow on a periodic box: the error
    after a fixed time decreases at least second order (RK2 in time)."""
    errs = []
    for n in (16, 32, 64):
        d = 1.0 / n
        mat = {"gamma": 1.4, "pinf": 0.0}
        cfg = inputs.config(n, 1, d, d, mat, mat, ["periodic"] * 2 + ["zerograd"] * 2, dim=1)
        x = (np.arange(n) + 0.5) * d
        rho = 1.0 + 0.2 * np.sin(2 * np.pi * x)
        pr = np.stack([rho, np.full(n, 1.0), np.zeros(n), np.full(n, 1.0)])[:, None, :]
        phi = np.ones((1, n))
        o = O.Oracle(cfg).init(phi, pr, pr)
        T = 0.25
        o.step_single_dt(100000, T)
        qN, qP, _ = o.state()
        exact = 1.0 + 0.2 * np.sin(2 * np.pi * (x - T))
        errs.append(np.abs(qP[0, 0] - exact).max())
    assert errs[1] < errs[0] / 3.5 and errs[2] < errs[1] / 3.5, errs
