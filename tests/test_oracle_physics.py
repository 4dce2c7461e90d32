"""Integration pins of the oracle: invariants that the method must satisfy
whatever the implementation (static interface, exact conservation with the
interfacial flux correction of Eq. 8-9, ratio-one reduction of the
multi-time-step cycle to the single-step method, mirror symmetry, the
exact 1D gas-water Riemann solution, rigid level-set translation)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs
from tests import exact_riemann as ER


def _pressure(q, alpha, g, pi):
    m = alpha > 1e-6
    a = np.where(m, alpha, 1.0)
    rho = q[0] / a
    q0 = np.where(q[0] != 0, q[0], 1.0)
    u, v = q[1] / q0, q[2] / q0
    p = (g - 1) * (q[3] / a - 0.5 * rho * (u * u + v * v)) - g * pi
    return p[m], u[m], v[m]


@pytest.mark.parametrize("multi", [False, True])
def test_static_interface_stays_static(multi):
    c = inputs.static_interface(32, 32)
    cfg = c["cfg"]
    o = O.Oracle(cfg).init(c["phi"], c["prim_N"], c["prim_P"])
    for _ in range(100):
        o.step_multi_dt(1) if multi else o.step_single_dt(1)
    assert o.status == 0
    qN, qP, _ = o.state()
    al = o.geometry()["alpha"]
    for k, q, a in ((0, qN, 1 - al), (1, qP, al)):
        p, u, v = _pressure(q, a, cfg["gamma"][k], cfg["pinf"][k])
        assert np.abs(p - 1e5).max() <= 1e-12 * (1e5 + cfg["pinf"][k])
        assert np.abs(u).max() <= 1e-12 and np.abs(v).max() <= 1e-12


def _drift(o, I0):
    I1 = o.integrals().sum(0)
    mass0, en0 = I0[0], I0[3]
    # momentum is compared with the mass times the largest speed in the box
    mscale = mass0 * 2000.0
    return np.array([abs(I1[0] - I0[0]) / mass0, abs(I1[1] - I0[1]) / mscale,
                     abs(I1[2] - I0[2]) / mscale, abs(I1[3] - I0[3]) / en0])


@pytest.mark.parametrize("seed", [1, 2])
def test_multi_dt_conserves_with_flux_correction(seed):
    c = inputs.periodic_bubble(48, seed=seed)
    o = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    I0 = o.integrals().sum(0)
    subs = []
    for _ in range(60):
        subs.append(o.step_multi_dt(1)["substeps"])
    assert o.status == 0
    assert max(subs) >= 2  # the gas sub-cycles
    assert _drift(o, I0).max() <= 1e-13


def test_multi_dt_without_correction_loses_conservation():
    c = inputs.periodic_bubble(48, seed=1)
    cfg = dict(c["cfg"], flux_correction=0)
    o = O.Oracle(cfg).init(c["phi"], c["prim_N"], c["prim_P"])
    I0 = o.integrals().sum(0)
    for _ in range(60):
        o.step_multi_dt(1)
    d = _drift(o, I0)
    assert d[0] <= 1e-13          # no mass crosses the interface
    assert max(d[1], d[2]) > 1e-8  # momentum exchange is no longer balanced


def test_single_dt_conserves():
    c = inputs.periodic_bubble(48, seed=3)
    o = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    I0 = o.integrals().sum(0)
    for _ in range(60):
        o.step_single_dt(1)
    assert o.status == 0 and _drift(o, I0).max() <= 1e-13


@pytest.mark.parametrize("case", ["bubble", "tube"])
def test_ratio_one_cycle_equals_single_step_bitwise(case):
    if case == "bubble":
        c = inputs.periodic_bubble(32, seed=4)
    else:
        c = inputs.shock_tube_1d(200, rk_order=2)
    a = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    b = O.Oracle(dict(c["cfg"], force_ratio_one=1)).init(c["phi"], c["prim_N"], c["prim_P"])
    for _ in range(25):
        a.step_single_dt(1)
        b.step_multi_dt(1)
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)
    assert a.t == b.t


def test_mirror_symmetry_of_shock_bubble():
    c = inputs.shock_bubble(128, 32)
    for multi in (False, True):
        o = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
        for _ in range(100):
            o.step_multi_dt(1) if multi else o.step_single_dt(1)
        assert o.status == 0
        qN, qP, phi = o.state()
        for q in (qN, qP):
            for m, sgn in ((0, 1), (1, 1), (2, -1), (3, 1)):
                asym = np.abs(q[m] - sgn * q[m][::-1, :]).sum() / max(np.abs(q[m]).sum(), 1e-300)
                scale = np.abs(q[0]).sum() if m == 2 else np.abs(q[m]).sum()
                asym = np.abs(q[m] - sgn * q[m][::-1, :]).sum() / max(scale, 1e-300)
                assert asym <= 1e-12
        assert np.abs(phi - phi[::-1, :]).max() <= 1e-12


def _tube_errors(n, rk, multi, T=2e-4, weno_char=0):
    c = inputs.shock_tube_1d(n, rk_order=rk)
    c["cfg"]["weno_char"] = weno_char
    o = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    while o.t < T * (1 - 1e-14):
        (o.step_multi_dt if multi else o.step_single_dt)(1, T)
    assert o.status == 0
    qN, qP, phi = o.state()
    d = 1.0 / n
    rho_mix = (qN[0, 0] + qP[0, 0])  # sum_k alpha_k rho_k per cell
    xs = (np.arange(n)[:, None] + (np.arange(16)[None, :] + 0.5) / 16) * d
    L = (1000.0, 0.0, 1.0e9, 4.4, 6.0e8)
    R = (1.0, 0.0, 1.0e5, 1.4, 0.0)
    ex, ps, us, xc = ER.sample_left_rarefaction_right_shock(L, R, 0.5, T, xs.ravel())
    ex = np.array(ex).reshape(n, 16).mean(axis=1)
    l1 = np.abs(rho_mix - ex).sum() * d
    f = phi[0]
    k = np.nonzero((f[:-1] < 0) & (f[1:] >= 0))[0][0]
    xi = (k + 0.5 + f[k] / (f[k] - f[k + 1])) * d
    return l1, abs(xi - xc) / d


@pytest.mark.parametrize("rk,multi", [(3, False), (2, False), (2, True)])
def test_shock_tube_converges_to_exact_solution(rk, multi):
    """L1 error of the mixture density against the cell-averaged exact
    solution falls at every refinement from 200 to 1600 cells (about first
    order at the discontinuities), and the contact sits within 2 cells."""
    errs, cons = zip(*(_tube_errors(n, rk, multi) for n in (200, 400, 800, 1600)))
    assert all(b < 0.8 * a for a, b in zip(errs, errs[1:])), errs
    assert max(cons) <= 2.0, cons


def test_level_set_rigid_translation():
    errs = []
    for n in (32, 64):
        d = 1.0 / n
        mat = {"gamma": 1.4, "pinf": 0.0}
        cfg = inputs.config(n, n, d, d, mat, mat, ["periodic"] * 4)
        X, Y = inputs._centres(cfg)
        R, u, v = 0.2, 100.0, 50.0
        phi = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2) - R
        pr = inputs._uniform(X.shape, 1.0, u, v, 1e5)
        o = O.Oracle(cfg).init(phi, pr, pr)
        T = 0.2 / math.hypot(u, v)
        o.step_single_dt(100000, T)
        assert o.status == 0
        area = (1 - o.geometry()["alpha"]).sum() * d * d
        errs.append(abs(area - math.pi * R * R) / (math.pi * R * R))
        qN, _, _ = o.state()
        rho = qN[0] / np.maximum(1 - o.geometry()["alpha"], 1e-300)
        m = (1 - o.geometry()["alpha"]) > 1e-6
        assert np.abs(rho[m] - 1.0).max() < 0.01
    assert errs[1] < errs[0] / 3.0 and errs[1] < 5e-3, errs


def test_reinitialisation_keeps_planar_distance():
    n = 32
    d = 1.0 / n
    mat = {"gamma": 1.4, "pinf": 0.0}
    cfg = inputs.config(n, n, d, d, mat, mat, ["periodic", "periodic", "reflect", "reflect"], band=1e9)
    X, Y = inputs._centres(cfg)
    phi = X - 0.513
    pr = inputs._uniform(X.shape, 1.0, 0.0, 0.0, 1.0)
    o = O.Oracle(cfg).init(phi, pr, pr)
    o.reinit_only()
    _, _, ph = o.state()
    inner = slice(4, n - 4)
    assert np.abs(ph[:, inner] - phi[:, inner]).max() <= 1e-14


def test_mixing_conserves_and_averages():
    c = inputs.periodic_bubble(32, seed=5)
    o = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    # perturb one small cut cell so that mixing has work to do
    qN, qP, phi = o.state()
    al = 1 - o.geometry()["alpha"]
    cand = np.argwhere((al > 1e-3) & (al < 0.2))
    j, i = cand[0]
    qN = qN.copy()
    qN[:, j, i] *= 3.0
    o.set_state(qN, qP, phi)
    before = o.integrals()
    o.mix_only(0)
    after = o.integrals()
    assert np.abs(after - before).max() <= 1e-15 * np.abs(before).max()
    qN2, _, _ = o.state()
    # the small cell's state is now a volume-weighted average: its density
    # lies between the densities of the cells it exchanged with
    rho = qN2[0, j, i] / al[j, i]
    assert 0.5 < rho < 3.0


def test_extension_reproduces_uniform_state():
    c = inputs.static_interface(32, 32)
    o = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    for k, ref in ((0, c["prim_N"]), (1, c["prim_P"])):
        W = o.stencil_states(k)
        assert np.abs(W - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("multi", [False, True])
def test_shock_bubble_runs_through_the_interaction(multi):
    """The Mach 1.22 shock through the helium bubble to t = 1.0 (the shock
    passes the bubble and the bubble rolls up into a kidney): no
    non-physical state, no spurious fluid-N region away from the bubble,
    and the helium volume stays within the compression the shock causes."""
    case = inputs.shock_bubble(128, 32)
    o = O.Oracle(case["cfg"]).init(case["phi"], case["prim_N"], case["prim_P"])
    area0 = float((case["phi"] < 0).sum())
    while o.t < 1.0:
        info = o.step_multi_dt(1) if multi else o.step_single_dt(1)
        assert info["err"] == 0, (o.t, info)
    qN, qP, phi = o.state()
    assert np.all(np.isfinite(qN)) and np.all(np.isfinite(qP))
    neg = phi < 0
    assert 0.3 * area0 < neg.sum() < area0
    # one helium region: every negative cell lies within 0.4 of the
    # negative region's centroid (the bubble has moved, not fragmented)
    X, Y = np.meshgrid(np.arange(128) * case["cfg"]["dx"], np.arange(32) * case["cfg"]["dy"])
    cx, cy = X[neg].mean(), Y[neg].mean()
    assert np.max(np.hypot(X[neg] - cx, Y[neg] - cy)) < 0.4


def _mixture(o):
    qN, qP, _ = o.state()
    return np.concatenate([(qN[0] + qP[0]).ravel(), (qN[3] + qP[3]).ravel()])


def test_multi_and_single_dt_meet_as_the_step_shrinks():
    """Both forms discretise the same semi-discrete system: at a fixed time
    their difference shrinks monotonically with the CFL number (the gas
    sub-cycles twice per water step in this tube)."""
    c = inputs.shock_tube_1d(400, rk_order=2)
    T = 1.0e-4
    diffs = []
    for cfl in (0.6, 0.3, 0.15, 0.075):
        cfg = dict(c["cfg"], cfl=cfl)
        runs = []
        for multi in (False, True):
            o = O.Oracle(cfg).init(c["phi"], c["prim_N"], c["prim_P"])
            subs = []
            while o.t < T * (1 - 1e-14):
                info = (o.step_multi_dt if multi else o.step_single_dt)(1, T)
                subs.append(info["substeps"])
            assert o.status == 0
            runs.append(_mixture(o))
            if multi:
                assert max(subs) >= 2
        diffs.append(np.abs(runs[1] - runs[0]).sum() / np.abs(runs[0]).sum())
    assert all(b < a for a, b in zip(diffs, diffs[1:])), diffs
    assert diffs[-1] < 0.3 * diffs[0], diffs


def test_mirror_symmetry_of_centred_explosion():
    """A gas bubble at the centre of a reflective box stays symmetric about
    both axes (x-momentum odd in x, y-momentum odd in y)."""
    c = inputs.underwater_explosion(64)
    for multi in (False, True):
        o = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
        for _ in range(40):
            o.step_multi_dt(1) if multi else o.step_single_dt(1)
        assert o.status == 0
        qN, qP, phi = o.state()
        for q in (qN, qP):
            mass = np.abs(q[0]).sum()
            for m, sx, sy in ((0, 1, 1), (1, -1, 1), (2, 1, -1), (3, 1, 1)):
                scale = max(np.abs(q[m]).sum(), mass if m in (1, 2) else 0.0, 1e-300)
                ax = np.abs(q[m] - sx * q[m][:, ::-1]).sum() / scale
                ay = np.abs(q[m] - sy * q[m][::-1, :]).sum() / scale
                assert ax <= 1e-12 and ay <= 1e-12, (multi, m, ax, ay)
        assert np.abs(phi - phi[:, ::-1]).max() <= 1e-12
        assert np.abs(phi - phi[::-1, :]).max() <= 1e-12


def test_reflective_box_conserves_mass_and_energy():
    """Walls exchange momentum but no mass or energy: the multi-time-step
    cycle with the correction keeps both totals of the two fluids."""
    c = inputs.underwater_explosion(48)
    o = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    I0 = o.integrals().sum(0)
    subs = [o.step_multi_dt(1)["substeps"] for _ in range(40)]
    assert o.status == 0 and max(subs) >= 2
    I1 = o.integrals().sum(0)
    assert abs(I1[0] - I0[0]) <= 1e-13 * abs(I0[0])
    assert abs(I1[3] - I0[3]) <= 1e-13 * abs(I0[3])
