"""Pins of the oracle's HLLC face flux (option flux = "hllc"; Toro's HLLC
with Davis's wave-speed bounds between WENO5 reconstructions of the
primitive state).  Flux level: consistency with the physical flux, exact
upwinding of supersonic states, the exact flux of stationary and moving
contacts, mirror and rotation symmetry, and agreement with the exact
Riemann solution of a weak acoustic problem to first order in its
amplitude.  Scheme level: a contact at rest inside one fluid stays exactly
at rest (the Lax-Friedrichs flux smears it), the Sod tube's error is below
the Lax-Friedrichs flux's at every resolution, conservation, and the
options the flux refuses."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs
from tests import exact_riemann as ER

IG = {"gamma": 1.4, "pinf": 0.0}


def phys(W, g, pi, d):
    """Euler flux of direction d of a primitive state (rho, u, v, p)."""
    r, u, v, p = W
    E = (p + g * pi) / (g - 1.0) + 0.5 * r * (u * u + v * v)
    un = u if d == 0 else v
    f = np.array([r * un, r * u * un, r * v * un, un * (E + p)])
    f[1 + d] += p
    return f


def test_consistency_with_the_physical_flux():
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(300):
        g = rng.uniform(1.1, 7.0)
        pi = 0.0 if rng.random() < 0.5 else rng.uniform(0.0, 10.0)
        W = [rng.uniform(0.1, 5.0), rng.normal(), rng.normal(), rng.uniform(0.1, 5.0)]
        for d in (0, 1):
            F, ref = O.hllc(W, W, g, pi, d), phys(W, g, pi, d)
            worst = max(worst, np.abs(F - ref).max() / np.abs(ref).max())
    assert worst < 1e-13


@pytest.mark.parametrize("d", [0, 1])
def test_supersonic_states_are_upwinded_exactly(d):
    g = 1.4
    fast = [3.0, 0.2] if d == 0 else [0.2, 3.0]
    WL, WR = [1.0, *fast, 1.0], [0.5, *[x * 0.95 for x in fast], 0.8]
    assert np.array_equal(O.hllc(WL, WR, g, 0.0, d), phys(WL, g, 0.0, d))
    mL = [WL[0], *[-x for x in fast], WL[3]]
    mR = [WR[0], *[-x * 0.95 for x in fast], WR[3]]
    assert np.array_equal(O.hllc(mL, mR, g, 0.0, d), phys(mR, g, 0.0, d))


@pytest.mark.parametrize("pinf", [0.0, 3.0])
@pytest.mark.parametrize("d", [0, 1])
def test_stationary_contact_gives_the_pressure_flux_only(pinf, d):
    """Different densities and tangential velocities, no normal velocity,
    equal pressure: the exact flux is the pressure on the normal momentum."""
    g, p = 4.4, 2.0
    t = [0.3, -0.5]
    WL = [1.0, 0.0, t[0], p] if d == 0 else [1.0, t[0], 0.0, p]
    WR = [0.1, 0.0, t[1], p] if d == 0 else [0.1, t[1], 0.0, p]
    F = O.hllc(WL, WR, g, pinf, d)
    ref = np.zeros(4)
    ref[1 + d] = p
    assert np.abs(F - ref).max() <= 1e-15 * p


@pytest.mark.parametrize("un", [0.3, -0.3])
def test_moving_contact_flux_is_the_upwind_physical_flux(un):
    g = 1.4
    WL, WR = [1.0, un, 0.2, 2.0], [0.1, un, -0.5, 2.0]
    F = O.hllc(WL, WR, g, 0.0, 0)
    ref = phys(WL if un > 0 else WR, g, 0.0, 0)
    assert np.abs(F - ref).max() <= 1e-14 * np.abs(ref).max()


def test_mirror_symmetry():
    """Reflecting x: the flux between mirrored states taken in swapped
    order is the mirrored flux with the transported quantities negated."""
    rng = np.random.default_rng(1)
    for _ in range(100):
        WL = [rng.uniform(0.2, 3.0), rng.normal(), rng.normal(), rng.uniform(0.2, 3.0)]
        WR = [rng.uniform(0.2, 3.0), rng.normal(), rng.normal(), rng.uniform(0.2, 3.0)]
        F = O.hllc(WL, WR, 1.4, 0.5, 0)
        mL, mR = [WR[0], -WR[1], WR[2], WR[3]], [WL[0], -WL[1], WL[2], WL[3]]
        G = O.hllc(mL, mR, 1.4, 0.5, 0)
        ref = np.array([-F[0], F[1], -F[2], -F[3]])
        assert np.abs(G - ref).max() <= 1e-13 * (1.0 + np.abs(F).max())


def test_y_flux_is_the_rotated_x_flux():
    rng = np.random.default_rng(2)
    for _ in range(100):
        WL = [rng.uniform(0.2, 3.0), rng.normal(), rng.normal(), rng.uniform(0.2, 3.0)]
        WR = [rng.uniform(0.2, 3.0), rng.normal(), rng.normal(), rng.uniform(0.2, 3.0)]
        Fx = O.hllc(WL, WR, 1.4, 0.0, 0)
        Fy = O.hllc([WL[0], WL[2], WL[1], WL[3]], [WR[0], WR[2], WR[1], WR[3]], 1.4, 0.0, 1)
        assert np.abs(Fy - Fx[[0, 2, 1, 3]]).max() <= 1e-14 * (1.0 + np.abs(Fx).max())


@pytest.mark.parametrize("amp", [1e-3, 1e-4])
def test_weak_acoustic_problem_matches_the_exact_solution(amp):
    """Equal densities, a small pressure step: the face lies in the exact
    solution's left star state (the contact moves right); HLLC's mass flux
    matches rho*_L u* to first order in the amplitude and its momentum flux
    p* + rho*_L u*^2 to second order."""
    g = 1.4
    L, R = (1.0, 0.0, 1.0 + amp), (1.0, 0.0, 1.0)
    ex = O.riemann((L[0], L[1], L[2], g, 0.0), (R[0], R[1], R[2], g, 0.0))
    F = O.hllc([L[0], L[1], 0.0, L[2]], [R[0], R[1], 0.0, R[2]], g, 0.0, 0)
    mass = ex["rho_L"] * ex["u"]
    assert abs(F[0] - mass) <= 0.5 * amp * abs(mass)
    assert abs(F[1] - (ex["p"] + ex["rho_L"] * ex["u"] ** 2)) <= 0.05 * amp * amp


def test_non_physical_states_are_refused():
    assert O.hllc([-1.0, 0, 0, 1.0], [1.0, 0, 0, 1.0], 1.4, 0.0, 0) is None
    assert O.hllc([1.0, 0, 0, 1.0], [1.0, 0, 0, -2.0], 1.4, 1.0, 0) is None


def _tube(n, flux, L, R, T, x_contact=None):
    d = 1.0 / n
    cfg = dict(inputs.config(n, 1, d, d, IG, IG, ["zerograd"] * 4, dim=1, rk_order=2),
               flux=flux)
    x = (np.arange(n) + 0.5) * d
    phi = (x - 0.5)[None, :]
    pN = inputs._uniform((1, n), L[0], L[1], 0.0, L[2])
    pP = inputs._uniform((1, n), R[0], R[1], 0.0, R[2])
    if x_contact is not None:
        pP[0][0, x > x_contact] *= 4.0
    o = O.Oracle(cfg).init(phi, pN, pP)
    while o.t < T:
        o.step_single_dt(1, t_end=T)
    return o


@pytest.mark.parametrize("n", [100, 200])
def test_sod_error_below_the_lax_friedrichs_flux(n):
    """Sod's problem (the two fluids the same ideal gas, the interface at
    the contact): relative L1 of the density against the exact solution,
    cell-averaged, at t = 0.2."""
    L, R, T = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.2
    xs = (np.arange(n)[:, None] + (np.arange(16)[None, :] + 0.5) / 16) / n
    ex, _, _, _ = ER.sample_left_rarefaction_right_shock(L + (1.4, 0.0), R + (1.4, 0.0), 0.5,
                                                         T, xs.ravel())
    ex = np.array(ex).reshape(n, 16).mean(axis=1)
    err = {}
    for flux in ("lf", "hllc"):
        qN, qP, _ = _tube(n, flux, L, R, T).state()
        err[flux] = np.abs(qN[0, 0] + qP[0, 0] - ex).sum() / n
    assert err["hllc"] < 0.85 * err["lf"], err
    assert err["hllc"] < 0.5 / n, err


def test_contact_at_rest_inside_a_fluid_stays_sharp():
    """A density jump at rest at x = 0.75 inside fluid P (uniform pressure,
    no velocity): HLLC keeps it to round-off; Lax-Friedrichs smears it."""
    L = R = (1.0, 0.0, 1.0)
    n = 64
    out = {}
    for flux in ("lf", "hllc"):
        o = _tube(n, flux, L, R, 0.3, x_contact=0.75)
        qN, qP, _ = o.state()
        out[flux] = qN[0, 0] + qP[0, 0]
    x = (np.arange(n) + 0.5) / n
    init = np.where(x > 0.75, 4.0, 1.0)
    assert np.abs(out["hllc"] - init).max() <= 1e-12
    assert np.abs(out["lf"] - init).max() >= 1e-2


def test_conservation_with_hllc():
    case = inputs.periodic_bubble(32, seed=3)
    o = O.Oracle(dict(case["cfg"], flux="hllc")).init(case["phi"], case["prim_N"],
                                                      case["prim_P"])
    before = o.integrals()
    o.step_single_dt(10)
    o.step_multi_dt(5)
    after = o.integrals()
    tot0 = before[0] + before[1]
    tot1 = after[0] + after[1]
    assert np.abs(tot1 - tot0).max() <= 1e-12 * np.abs(tot0).max()


def test_hllc_with_characteristic_reconstruction_is_refused():
    case = inputs.periodic_bubble(16, seed=3)
    with pytest.raises(Exception):
        O.Oracle(dict(case["cfg"], flux="hllc", weno_char=1))
    with pytest.raises(ValueError):
        O.Oracle(dict(case["cfg"], flux="roe"))
