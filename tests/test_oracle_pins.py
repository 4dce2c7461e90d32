"""Pins of oracle parts that the physics tests leave loose: the ghost-state
extension (Sec. 2.3), the sum form of the CFL rate and the star speed in
it (Sec. 2.3 "according to CFL conditions"; the reading with the
interface star state), and the choice of small-cell mixing targets
(Sec. 2.2).  Each test is built so that a plausible mistake in the oracle
-- a sweep taking the downwind neighbour, the wrong sign of the fluid
normal, a max instead of the sum of the directional rates, a dropped
star speed, mixing toward the other fluid -- fails it."""
import math

import numpy as np

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs

from tests import exact_riemann as ER

GAS = {"gamma": 1.4, "pinf": 0.0}


def _garbage(rng, shape):
    """Physical but unrelated primitive states (rho, u, v, p)."""
    g = np.empty((4,) + shape)
    g[0] = rng.uniform(0.5, 2.0, shape)
    g[1] = rng.uniform(-1.0, 1.0, shape)
    g[2] = rng.uniform(-1.0, 1.0, shape)
    g[3] = rng.uniform(0.5, 2.0, shape)
    return g


def _linear_state(T):
    """A state that is linear in the tangential coordinate T."""
    return np.stack([1.0 + 0.5 * T, 0.1 + 0.2 * T, -0.05 + 0.1 * T, 1.0 + 0.3 * T])


def _conserved(w, gamma=1.4):
    rho, u, v, p = w
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def _extension_case(n, angle):
    cfg = inputs.config(n, n, 1.0 / n, 1.0 / n, GAS, GAS, ["zerograd"] * 4)
    X, Y = inputs._centres(cfg)
    nx_, ny_ = math.cos(angle), math.sin(angle)
    # the interface crosses the cells off their faces and centres
    phi = (X - 0.5) * nx_ + (Y - 0.5) * ny_ - 0.3 / n
    T = -(X - 0.5) * ny_ + (Y - 0.5) * nx_   # tangential coordinate
    return cfg, phi, T


def test_extension_reproduces_tangentially_linear_fields_from_the_fluid_side():
    """n_k . grad W = 0 holds exactly for a field that is constant along the
    normal, and the upwind sweeps reproduce a field linear in the
    tangential coordinate exactly (grid-aligned interface: each target
    copies its neighbour toward the fluid; 45 degrees: the mean of its two
    neighbours toward the fluid, whose linear parts cancel).  Fluid N's
    initial states beyond the interface are unrelated random values: a
    sweep that reads the downwind neighbour, or takes the normal with the
    wrong sign, carries them into the band instead."""
    rng = np.random.default_rng(11)
    n = 32
    h = 1.0 / n
    for angle in (0.0, math.pi / 4):
        cfg, phi, T = _extension_case(n, angle)
        lin = _linear_state(T)
        pN = np.where(phi > 1.5 * h, _garbage(rng, phi.shape), lin)
        pP = inputs._uniform(phi.shape, 1.0, 0.0, 0.0, 1.0)
        o = O.Oracle(cfg).init(phi, pN, pP)
        # the real cells hold the linear field exactly: set the conserved
        # state without the initial mixing (which averages neighbours of
        # different tangential coordinate); the extension starts from pN
        al = o.geometry()["alpha"]
        o.set_state((1.0 - al) * _conserved(lin), al * _conserved(pP), phi)
        W = o.stencil_states(0)
        near = (phi > 0.0) & (phi < 4.0 * h)
        # cells whose normal (central differences of phi) reads ghost
        # values of the zero-gradient walls have a tilted normal: leave
        # them out
        near[[0, -1], :] = False
        near[:, [0, -1]] = False
        assert near.sum() > 3 * n
        err = np.abs(W[:, near] - lin[:, near]).max()
        assert err <= 1e-13, (angle, err)
        # outside the band nothing is extended: the initial values stay
        far = phi > 6.5 * h
        assert np.array_equal(W[:, far], pN[:, far])


def test_cfl_step_of_a_uniform_moving_state_is_the_sum_form():
    """dt = CFL / ((|u| + c)/dx + (|v| + c)/dy) for a uniform state in a
    periodic box of one fluid (dx != dy; a max of the two rates instead of
    their sum gives a step about twice as long)."""
    nx, ny = 24, 16
    cfg = inputs.config(nx, ny, 1.0 / nx, 1.0 / ny, GAS, GAS, ["periodic"] * 4)
    phi = np.ones((ny, nx))
    rho, u, v, p = 1.3, 0.7, -0.4, 2.1
    pP = inputs._uniform((ny, nx), rho, u, v, p)
    o = O.Oracle(cfg).init(phi, pP.copy(), pP)
    info = o.step_single_dt(1)
    c = math.sqrt(1.4 * p / rho)
    expect = 0.6 / ((abs(u) + c) * nx + (abs(v) + c) * ny)
    assert abs(info["dt1"] - expect) <= 1e-14 * expect


def test_tube_time_step_ratio_includes_the_air_star_speed():
    """In the water/air tube at rest the air's CFL rate is set by its star
    state at the interface (|u*| + c*_air = 985 m/s against c_air = 374
    m/s), the water's by its sound speed (2653 m/s): the first cycle's
    ratio n = dt_air / dt_water is c_water / (|u*| + c*_air), with the star
    state from an independent exact solver.  Without the star speed n
    would be 7.09."""
    c = inputs.shock_tube_1d(400, rk_order=2)
    o = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    info = o.step_multi_dt(1)
    L = (1000.0, 0.0, 1.0e9, 4.4, 6.0e8)
    R = (1.0, 0.0, 1.0e5, 1.4, 0.0)
    ps, us = ER.star_state(L, R)
    rho_air = ER.hugoniot_density(ps, 1.0, 1.0e5, 1.4, 0.0)
    c_air_star = math.sqrt(1.4 * ps / rho_air)
    c_water = math.sqrt(4.4 * (1.0e9 + 6.0e8) / 1000.0)
    expect = c_water / (abs(us) + c_air_star)
    assert info["role_fluid1"] == 1               # air (fluid P) takes the larger step
    assert abs(info["n_raw"] - expect) <= 1e-9 * expect, (info["n_raw"], expect)


def _mix_case(n, phi, U0, src_mask, U1):
    """Fluid P holding state U0 everywhere except the cells of src_mask,
    which hold U1 (conserved variables per unit volume)."""
    cfg = inputs.config(n, n, 1.0 / n, 1.0 / n, GAS, GAS, ["reflect"] * 4)
    pP = inputs._uniform(phi.shape, 1.0, 0.0, 0.0, 1.0)
    o = O.Oracle(cfg).init(phi, pP.copy(), pP)
    al = o.geometry()["alpha"]
    qP = np.where(src_mask, al * U1[:, None, None], al * U0[:, None, None])
    qN = np.zeros_like(qP)
    o.set_state(qN, qP, phi)
    return o, al, qP


def test_mixing_toward_the_fluid_averages_with_the_cell_above():
    """Horizontal interface, fluid P above: the small P cells of the
    interface row (alpha_P = 0.3) have one mixing target, the cell above
    them (the normal points straight into the fluid), and pairwise
    volume-weighted mixing leaves both cells of each pair at the pair's
    volume-weighted mean state.  Mixing toward the other fluid would pick
    an empty cell below, be refused, and move content sideways instead."""
    n = 8
    h = 1.0 / n
    X, Y = np.meshgrid((np.arange(n) + 0.5) * h, (np.arange(n) + 0.5) * h)
    phi = Y - 3.7 * h
    U0 = np.array([1.0, 0.2, -0.1, 2.5])
    U1 = np.array([1.6, -0.3, 0.4, 3.1])
    src = np.zeros((n, n), bool)
    src[3, :] = True
    o, al, q0 = _mix_case(n, phi, U0, src, U1)
    assert np.allclose(al[3], 0.3, atol=1e-14) and np.all(al[4:] == 1.0) and np.all(al[:3] == 0.0)
    o.mix_only(1)
    _, q, _ = o.state()
    a3 = al[3, 0]
    mean = (a3 * U1 + U0) / (a3 + 1.0)
    assert np.abs(q[:, 3, :] / a3 - mean[:, None]).max() <= 1e-14
    assert np.abs(q[:, 4, :] - mean[:, None]).max() <= 1e-14
    # nothing else moved
    others = np.ones(n, bool)
    others[[3, 4]] = False
    assert np.array_equal(q[:, others, :], q0[:, others, :])


def test_mixing_at_45_degrees_uses_the_three_cells_toward_the_fluid():
    """Interface x + y = c, fluid P toward +x +y: a small P cell exchanges
    with its +x, +y and diagonal neighbours (weights n_x^2, n_y^2,
    |n_x n_y|, equal here), and nothing else; by the mirror symmetry of
    the configuration about the diagonal the +x and +y neighbours receive
    the same amounts; the exchange conserves every component."""
    n = 12
    h = 1.0 / n
    X, Y = np.meshgrid((np.arange(n) + 0.5) * h, (np.arange(n) + 0.5) * h)
    phi = (X + Y - 11.1 * h) / math.sqrt(2.0)
    cfg = inputs.config(n, n, h, h, GAS, GAS, ["reflect"] * 4)
    probe = O.Oracle(cfg).init(phi, inputs._uniform(phi.shape, 1.0, 0.0, 0.0, 1.0),
                               inputs._uniform(phi.shape, 1.0, 0.0, 0.0, 1.0))
    al = probe.geometry()["alpha"]
    # a small P cell on the diagonal whose three targets are not small
    cands = [(j, i) for j in range(1, n - 1) for i in range(1, n - 1)
             if i == j and 0.0 < al[j, i] < 0.5 and al[j, i + 1] >= 0.5
             and al[j + 1, i] >= 0.5 and al[j + 1, i + 1] >= 0.5]
    assert cands
    j, i = cands[0]
    src = np.zeros((n, n), bool)
    src[j, i] = True
    U0 = np.array([1.0, 0.2, 0.2, 2.5])
    U1 = np.array([1.6, -0.3, -0.3, 3.1])
    o, al, q0 = _mix_case(n, phi, U0, src, U1)
    o.mix_only(1)
    _, q, _ = o.state()
    d = q - q0
    changed = {(jj, ii) for jj, ii in zip(*np.nonzero(np.abs(d).max(axis=0) > 0.0))}
    assert changed == {(j, i), (j, i + 1), (j + 1, i), (j + 1, i + 1)}, changed
    assert np.abs(d[:, j, i + 1] - d[:, j + 1, i]).max() <= 1e-15
    assert np.abs(d.sum(axis=(1, 2))).max() <= 1e-15
    # content flows from the source to the targets along the difference
    # U0 - U1 of the states (every target gains U1 - U0 in proportion)
    for jj, ii in [(j, i + 1), (j + 1, i), (j + 1, i + 1)]:
        r = d[:, jj, ii] / (U1 - U0)
        assert np.all(r > 0.0) and np.ptp(r) <= 1e-12 * r.max()


# a level set (in cell sizes) whose cell (3, 3) is a small cell of fluid P
# with every neighbour along its normal small too, while the diagonal cell
# (4, 4), on the far side, is the only large one among its eight
# neighbours (found by a seeded search over random cell values)
FALLBACK_PHI = [
    [0.9552, 0.6392, 0.3317, -0.8522, -0.9501, -0.5694, 0.4804],
    [0.4172, 0.4063, -0.8709, -0.7265, 0.916, -0.0814, -0.1751],
    [-0.5485, 0.6076, 0.4587, -0.5417, -0.9063, -0.5847, -0.299],
    [0.5248, -0.3328, -0.649, 0.608, -0.7226, -0.9753, 0.5237],
    [0.0857, -0.5202, -0.5325, -0.8012, 0.9313, 0.2032, -0.8916],
    [-0.214, -0.6107, -0.0544, 0.8527, -0.4416, -0.2559, -0.9489],
    [-0.1315, -0.3844, -0.4929, 0.301, -0.3898, -0.8517, -0.2369]]


def test_mixing_falls_back_to_the_largest_of_the_eight_neighbours():
    """Reading 8's second rule: a small cell none of whose neighbours along
    its normal is large mixes with the largest of its eight neighbours when
    that one is large, even on the far side of the normal.  The source's
    state after mixing is then its own plus the exchange with that target,
    M = (q_t a_s - q_s a_t) / (a_s + a_t), both from the pre-mix states."""
    n = 7
    phi = np.array(FALLBACK_PHI) / n
    cfg = inputs.config(n, n, 1.0 / n, 1.0 / n, {"gamma": 1.4, "pinf": 0.0},
                        {"gamma": 1.4, "pinf": 0.0}, ["reflect"] * 4)
    o = O.Oracle(cfg)
    w = inputs._uniform((n, n), 1.0, 0.0, 0.0, 1.0)
    o.init(phi, w, w)
    a = o.geometry()["alpha"]
    i, j = 3, 3
    # the preconditions, from the oracle's geometry: a small source, its
    # normal's neighbours (x, y and diagonal, by the central-difference
    # gradient of phi) all small, and one large neighbour of the eight
    gx, gy = phi[j, i + 1] - phi[j, i - 1], phi[j + 1, i] - phi[j - 1, i]
    sx, sy = (1 if gx >= 0 else -1), (1 if gy >= 0 else -1)
    assert 0.0 < a[j, i] < 0.5
    for (ii, jj) in ((i + sx, j), (i, j + sy), (i + sx, j + sy)):
        assert a[jj, ii] < 0.5
    large = [(ii, jj) for jj in (j - 1, j, j + 1) for ii in (i - 1, i, i + 1)
             if (ii, jj) != (i, j) and a[jj, ii] >= 0.5]
    assert large == [(4, 4)] and (sx, sy) == (-1, -1)
    rng = np.random.default_rng(11)
    qP = np.stack([a * rng.uniform(0.5, 2.0, size=(n, n)) for _ in range(4)])
    o.set_state(np.zeros((4, n, n)).ravel(), qP.ravel(), phi.ravel())
    o.mix_only(1)
    out = o.state()[1][:, j, i]
    aS, aT = a[j, i], a[4, 4]
    expect = qP[:, j, i] + (qP[:, 4, 4] * aS - qP[:, j, i] * aT) / (aS + aT)
    assert np.abs(out - expect).max() <= 1e-14 * np.abs(expect).max()
    # what the other rules would have given differs: the normal's small
    # neighbours larger than the source (third rule), each alone
    for (ii, jj) in ((i - 1, j), (i - 1, j - 1)):
        aT = a[jj, ii]
        other = qP[:, j, i] + (qP[:, jj, ii] * aS - qP[:, j, i] * aT) / (aS + aT)
        assert np.abs(out - other).max() > 1e-3 * np.abs(expect).max()


# a small cell of fluid P at (3, 3) none of whose eight neighbours is large,
# two of its three neighbours along the normal larger than itself (found
# by a seeded search)
LARGER_PHI = [
    [0.459, 0.1005, -0.3754, 0.6933, -0.5151, -0.9433, 0.6208],
    [-0.4813, -0.2628, -0.8927, -0.9472, 0.3934, -0.0881, -0.1716],
    [0.2845, -0.4022, -0.29, -0.8526, -0.1154, -0.9, -0.9968],
    [-0.275, -0.8849, -0.2323, -0.3196, 0.7491, -0.4147, -0.6388],
    [-0.4156, 0.0833, -0.8958, 0.3905, -0.3218, -0.206, -0.4018],
    [-0.3836, -0.8128, -0.7969, 0.1585, -0.7968, -0.3252, -0.5658],
    [0.7711, -0.1644, -0.8841, -0.1825, -0.9758, -0.7902, 0.4431]]


def test_mixing_falls_back_to_larger_neighbours_along_the_normal():
    """Reading 8's third rule: with no large cell among the eight, the
    source mixes with the neighbours along its normal (x, y, diagonal, by
    the central-difference gradient of phi) that are larger than itself,
    with weights n_x^2, n_y^2, |n_x n_y| normalised over those kept:
    M_t = beta_t (q_t a_s - q_s a_t) / (a_s beta_t + a_t)."""
    n = 7
    phi = np.array(LARGER_PHI) / n
    cfg = inputs.config(n, n, 1.0 / n, 1.0 / n, {"gamma": 1.4, "pinf": 0.0},
                        {"gamma": 1.4, "pinf": 0.0}, ["reflect"] * 4)
    o = O.Oracle(cfg)
    w = inputs._uniform((n, n), 1.0, 0.0, 0.0, 1.0)
    o.init(phi, w, w)
    a = o.geometry()["alpha"]
    i, j = 3, 3
    assert 0.0 < a[j, i] < 0.5
    assert max(a[j + dj, i + di] for dj in (-1, 0, 1) for di in (-1, 0, 1)
               if (di, dj) != (0, 0)) < 0.5
    gx, gy = phi[j, i + 1] - phi[j, i - 1], phi[j + 1, i] - phi[j - 1, i]
    nx_, ny_ = gx / math.hypot(gx, gy), gy / math.hypot(gx, gy)
    sx, sy = (1 if nx_ >= 0 else -1), (1 if ny_ >= 0 else -1)
    cand = [((i + sx, j), nx_ * nx_), ((i, j + sy), ny_ * ny_), ((i + sx, j + sy), abs(nx_ * ny_))]
    kept = [(c, wt) for c, wt in cand if wt > 0 and a[c[1], c[0]] > a[j, i]]
    assert [c for c, _ in kept] == [(4, 3), (4, 4)]
    rng = np.random.default_rng(12)
    qP = np.stack([a * rng.uniform(0.5, 2.0, size=(n, n)) for _ in range(4)])
    o.set_state(np.zeros((4, n, n)).ravel(), qP.ravel(), phi.ravel())
    o.mix_only(1)
    out = o.state()[1][:, j, i]
    aS, W = a[j, i], sum(wt for _, wt in kept)
    expect = qP[:, j, i].copy()
    for (ti, tj), wt in kept:
        b, aT = wt / W, a[tj, ti]
        expect += b * (qP[:, tj, ti] * aS - qP[:, j, i] * aT) / (aS * b + aT)
    assert np.abs(out - expect).max() <= 1e-14 * np.abs(expect).max()
