"""Independent exact solution of the two-material stiffened-gas Riemann
problem, used to pin the oracle (tests only).

It is derived differently from the oracle's solver: the shock branch uses
the Rankine-Hugoniot mass flux m^2 = (p - p_K)/(1/rho_K - 1/rho*) with the
Hugoniot density of a stiffened gas, the rarefaction branch integrates
dp/(rho c) along the isentrope numerically, and the star pressure is
bracketed with Brent's method instead of Newton's.
"""
from __future__ import annotations

import math

from scipy.integrate import quad
from scipy.optimize import brentq


def hugoniot_density(p, rho, pk, g, pi):
    r = (p + pi) / (pk + pi)
    return rho * ((g + 1.0) * r + (g - 1.0)) / ((g - 1.0) * r + (g + 1.0))


def velocity_jump(p, rho, pk, g, pi):
    """u-change across the wave of side K (positive when p > p_K)."""
    if p > pk:
        rs = hugoniot_density(p, rho, pk, g, pi)
        m = math.sqrt((p - pk) / (1.0 / rho - 1.0 / rs))
        return (p - pk) / m

    def integrand(s):
        rs = rho * ((s + pi) / (pk + pi)) ** (1.0 / g)
        cs = math.sqrt(g * (s + pi) / rs)
        return 1.0 / (rs * cs)

    val, _ = quad(integrand, p, pk, epsabs=0.0, epsrel=1e-13, limit=200)
    return -val


def star_state(L, R):
    """L, R = (rho, u, p, gamma, pinf); returns p*, u*."""
    rl, ul, pl, gl, pil = L
    rr, ur, pr, gr, pir = R

    def F(p):
        return velocity_jump(p, rl, pl, gl, pil) + velocity_jump(p, rr, pr, gr, pir) + (ur - ul)

    lo = -min(pil, pir) + 1e-9 * min(pl + pil, pr + pir)
    hi = max(pl, pr) * 10.0 + 1.0
    while F(hi) < 0.0:
        hi *= 10.0
    p = brentq(F, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (velocity_jump(p, rr, pr, gr, pir) - velocity_jump(p, rl, pl, gl, pil))
    return p, us


def star_state_jump(L, R, jump):
    """As star_state with the left star pressure exceeding the right one by
    jump (a surface-tension pressure jump): returns the right star pressure
    p*, u*; the left star pressure is p* + jump."""
    rl, ul, pl, gl, pil = L
    rr, ur, pr, gr, pir = R

    def F(p):
        return (velocity_jump(p + jump, rl, pl, gl, pil) + velocity_jump(p, rr, pr, gr, pir)
                + (ur - ul))

    lo = max(-pir, -pil - jump) + 1e-9 * min(pl + pil, pr + pir)
    hi = max(pl, pr) * 10.0 + abs(jump) + 1.0
    while F(hi) < 0.0:
        hi *= 10.0
    p = brentq(F, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (velocity_jump(p, rr, pr, gr, pir)
                                  - velocity_jump(p + jump, rl, pl, gl, pil))
    return p, us


def sample_left_rarefaction_right_shock(L, R, x0, t, x):
    """Density at positions x (iterable) for a left rarefaction / right
    shock wave pattern; returns (rho(x) list, p*, u*, contact position)."""
    rl, ul, pl, gl, pil = L
    rr, ur, pr, gr, pir = R
    ps, us = star_state(L, R)
    assert ps < pl and ps > pr, "wave pattern is not rarefaction | shock"
    cl = math.sqrt(gl * (pl + pil) / rl)
    rsl = rl * ((ps + pil) / (pl + pil)) ** (1.0 / gl)
    csl = math.sqrt(gl * (ps + pil) / rsl)
    rsr = hugoniot_density(ps, rr, pr, gr, pir)
    S = (rsr * us - rr * ur) / (rsr - rr)
    head, tail = ul - cl, us - csl
    out = []
    for xi in x:
        s = (xi - x0) / t
        if s <= head:
            out.append(rl)
        elif s <= tail:
            c = 2.0 / (gl + 1.0) * (cl + 0.5 * (gl - 1.0) * (ul - s))
            out.append(rl * (c / cl) ** (2.0 / (gl - 1.0)))
        elif s <= us:
            out.append(rsl)
        elif s <= S:
            out.append(rsr)
        else:
            out.append(rr)
    return out, ps, us, x0 + us * t


def tait_density(p, B, rho0, p0, g):
    """Density on Tait's curve p = B ((rho/rho0)^g - 1) + p0."""
    return rho0 * ((p - p0) / B + 1.0) ** (1.0 / g)


def velocity_jump_tait(p, pk, B, rho0, p0, g):
    """u-change across the wave of a barotropic (Tait) side at star
    pressure p: a shock carries mass flux m with m^2 = (p - pk)/(1/rho_k -
    1/rho*) from mass and momentum alone; a rarefaction integrates
    dp/(rho c) along the curve, c^2 = dp/drho = g B rho^(g-1) / rho0^g."""
    rk = tait_density(pk, B, rho0, p0, g)
    if p > pk:
        rs = tait_density(p, B, rho0, p0, g)
        m = math.sqrt((p - pk) / (1.0 / rk - 1.0 / rs))
        return (p - pk) / m

    def integrand(s):
        r = tait_density(s, B, rho0, p0, g)
        c = math.sqrt(g * B * r ** (g - 1.0) / rho0 ** g)
        return 1.0 / (r * c)

    val, _ = quad(integrand, p, pk, epsabs=0.0, epsrel=1e-13, limit=200)
    return -val


def star_state_tait(L, R, pmin):
    """L, R = (u, p, jump_fn) per side, where jump_fn(p, pk) gives the
    side's u-change (velocity_jump_tait or velocity_jump bound to the
    side's parameters); pmin: the smallest pressure both sides admit (a
    Tait fluid's p0 - B, a stiffened gas's -p_inf); returns p*, u*."""
    ul, pl, fl = L
    ur, pr, fr = R

    def F(p):
        return fl(p, pl) + fr(p, pr) + (ur - ul)

    lo = pmin + 1e-9 * (min(pl, pr) - pmin)
    hi = max(pl, pr) * 10.0 + 1.0
    assert F(lo) < 0.0, "no star state above the admissible pressure"
    while F(hi) < 0.0:
        hi *= 10.0
    p = brentq(F, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (fr(p, pr) - fl(p, pl))
    return p, us
