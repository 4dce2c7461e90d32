"""Pins of the oracle's viscous fluxes (Eq. 3 and 5: central-difference
viscous face fluxes times the apertures, each fluid's viscous traction on
its interface boundary; part of the weakly compressible model of Sec. 2.2,
built here on the stiffened-gas equations) against closed forms of the
compressible Navier-Stokes equations with Stokes' hypothesis and no heat
conduction:
a shear wave decays as exp(-nu k^2 t) (in either orientation: the
x-face and y-face stresses), a standing sound wave as exp(-(2/3) nu k^2 t)
(the normal stresses with their 4/3 and 2/3), and the explicit viscous
time-step limit keeps a strongly viscous wave stable."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs

K2 = (2 * math.pi) ** 2


def _shear(n, across="y", mu=0.01, T=0.5, amp=0.01):
    c = inputs.shear_wave(n, mu=mu, amp=amp, across=across)
    o = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    I0 = o.integrals()
    while o.t < T * (1 - 1e-14):
        o.step_single_dt(1, T)
    assert o.status == 0
    _, qP, _ = o.state()
    x = (np.arange(n) + 0.5) / n
    if across == "y":
        a = 2.0 * ((qP[1] / qP[0]) * np.sin(2 * np.pi * x)[:, None]).mean()
    else:
        a = 2.0 * ((qP[2] / qP[0]) * np.sin(2 * np.pi * x)[None, :]).mean()
    return a / (amp * math.exp(-mu * K2 * T)) - 1.0, I0, o.integrals()


@pytest.mark.parametrize("across", ["y", "x"])
def test_shear_wave_decays_at_the_viscous_rate(across):
    e32, I0, I1 = _shear(32, across)
    e64, _, _ = _shear(64, across)
    assert abs(e32) < 1e-3 and abs(e64) < abs(e32) / 3.0, (e32, e64)
    # viscous fluxes are conservative: energy (heat gained = kinetic energy
    # lost) and the zero-mean momentum stay
    assert abs(I1[1, 3] / I0[1, 3] - 1.0) <= 1e-13
    assert abs(I1[1, 1]) + abs(I1[1, 2]) <= 1e-15 * I0[1, 0]


def test_without_viscosity_the_shear_wave_does_not_decay():
    e, _, _ = _shear(32, mu=0.0)
    assert abs(e) < 0.01


def test_explicit_viscous_limit_keeps_a_strongly_viscous_wave_stable():
    # nu = 1 on 32 cells: the acoustic step alone (nu dt / dx^2 = 0.8) would
    # exceed the explicit diffusion limit and the wave would blow up
    e, _, _ = _shear(32, mu=1.0, T=0.02)
    assert abs(e) < 0.02, e


def _sound_amplitude(n, mu, periods=4):
    c = inputs.sound_wave(n, mu=mu)
    o = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    T = periods / math.sqrt(1.4 * 100.0)  # whole periods: u returns to its shape
    while o.t < T * (1 - 1e-14):
        o.step_single_dt(1, T)
    assert o.status == 0
    _, qP, _ = o.state()
    x = (np.arange(n) + 0.5) / n
    return 2.0 * ((qP[1][0] / qP[0][0]) * np.sin(2 * np.pi * x)).mean(), T


def test_sound_wave_is_damped_by_the_normal_stresses():
    # the viscous run against the inviscid one isolates the viscous damping
    mu = 0.02
    for n in (64,):
        a_v, T = _sound_amplitude(n, mu)
        a_0, _ = _sound_amplitude(n, 0.0)
        ratio = a_v / a_0
        exact = math.exp(-(2.0 / 3.0) * mu * K2 * T)
        assert abs(ratio / exact - 1.0) < 2e-3, (ratio, exact)


def _rayleigh(n, muN, muP, T=0.5, U=0.1, m=4):
    """Fluid P sliding at U over fluid N at rest, the same gas on both
    sides, a flat interface 0.3 of a cell above y = 1/2 (reflective walls
    at y = 0, 1, periodic in x).  Returns fluid N's x momentum per unit
    length at T against the closed form, and the totals before and after."""
    d = 1.0 / n
    cfg = inputs.config(m, n, d, d, inputs.AIR, inputs.AIR,
                        ["periodic", "periodic", "reflect", "reflect"], mu=(muN, muP))
    X, Y = inputs._centres(cfg)
    phi = Y - (0.5 + 0.3 * d)
    pN = inputs._uniform(X.shape, 1.0, 0.0, 0.0, 100.0)
    pP = inputs._uniform(X.shape, 1.0, U, 0.0, 100.0)
    o = O.Oracle(cfg).init(phi, pN, pP)
    I0 = o.integrals()
    while o.t < T * (1 - 1e-14):
        o.step_single_dt(1, T)
    assert o.status == 0
    I1 = o.integrals()
    # two semi-infinite layers of equal density: the interface takes the
    # velocity U e_P / (e_N + e_P), e_k = sqrt(mu_k), and fluid N's
    # momentum is that velocity times 2 sqrt(nu_N t / pi)
    eN, eP = math.sqrt(muN), math.sqrt(muP)
    exact = U * eP / (eN + eP) * 2.0 * math.sqrt(muN * T / math.pi)
    return I1[0, 1] / (m * d) / exact - 1.0, I0, I1


@pytest.mark.parametrize("mus", [(0.01, 0.01), (0.01, 0.04)])
def test_interface_transmits_shear(mus):
    """The viscous traction across the interface couples the two fluids
    without slip: the momentum fluid N takes from fluid P sliding over it
    follows the two-layer diffusion solution (first order in the cell
    size at the interface: 3 % off at 128 cells), while momentum and
    energy only move between the fluids."""
    e64, _, _ = _rayleigh(64, *mus)
    e128, I0, I1 = _rayleigh(128, *mus)
    assert abs(e128) < 0.05 and abs(e128) < abs(e64) and abs(e64) < 0.1, (e64, e128)
    tot0, tot1 = I0.sum(axis=0), I1.sum(axis=0)
    assert abs(tot1[1] - tot0[1]) <= 1e-13 * abs(tot0[3])
    assert abs(tot1[3] / tot0[3] - 1.0) <= 1e-13
