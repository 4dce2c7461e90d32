"""Pins of the oracle's discrete adjoint of the frozen single-time-step
RK2 step (and of the initialisation), by means other than the adjoint code
itself: central finite differences of the forward functions, a brute-force
Jacobian on a tiny grid, exact transposition of the linear mixing, and the
conservation identities that the transposed step must satisfy exactly.

The gradient checks run in nondimensional gas-water units (states of order
one): WENO5-JS's epsilon is an absolute floor on the smoothness indicators,
so with SI-sized fluxes (~1e9) its weights vary on scales far below any
usable difference step and central differences of the forward map cannot
converge."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs


def _state(o):
    qN, qP, _ = o.state()
    return np.stack([qN, qP])


def test_weno5_grad_matches_central_differences():
    rng = np.random.default_rng(0)
    vecs = [rng.normal(size=5) for _ in range(6)]
    vecs += [np.array([1.0, 1.0, 1.0, 0.0, 0.0]), np.sin(np.arange(5) * 0.3),
             np.array([0.1, 0.2, 0.35, 0.45, 0.6])]
    for v in vecs:
        g = O.weno5_grad(v)
        h = 1e-6
        fd = np.array([(O.weno5(v + h * e) - O.weno5(v - h * e)) / (2 * h) for e in np.eye(5)])
        assert np.max(np.abs(g - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd)))
    # smooth limit: ideal weights, the derivative is the fifth-order stencil
    g = O.weno5_grad(np.full(5, 3.0))
    ideal = np.array([2.0, -13.0, 47.0, 27.0, -3.0]) / 60.0
    assert np.allclose(g, ideal, rtol=0, atol=1e-14)


RIEMANN_CASES = [
    ((1.0, 0.0, 1.0, 1.4, 0.0), (0.125, 0.0, 0.1, 1.4, 0.0)),          # shock + rarefaction
    ((1.0, -2.0, 0.4, 1.4, 0.0), (1.0, 2.0, 0.4, 1.4, 0.0)),            # two rarefactions
    ((1.0, 3.0, 1.0, 1.4, 0.0), (1.0, -3.0, 1.0, 1.4, 0.0)),            # two shocks
    ((1.0, 0.0, 1.0, 4.4, 0.6), (1.27e-3, 0.0, 1e-4, 1.4, 0.0)),        # water | gas
    ((1.27, 5e-3, 0.829, 1.4, 0.0), (1.0, -3e-3, 1e-4, 4.4, 0.6)),      # gas | water
]


@pytest.mark.parametrize("L,R", RIEMANN_CASES)
def test_riemann_grad_matches_central_differences(L, R):
    lam_p, lam_u = 0.7, -1.3

    def F(a, b):
        r = O.riemann(a, b)
        return lam_p * r["p"] + lam_u * r["u"]

    gL, gR = O.riemann_grad(L, R, lam_p, lam_u)
    got = np.concatenate([gL, gR])
    fd = []
    for side in (0, 1):
        for idx in (0, 1, 2):
            a, b = [list(L), list(R)], [list(L), list(R)]
            h = 1e-6 * max(abs(a[side][idx]), 1e-3)
            a[side][idx] += h
            b[side][idx] -= h
            fd.append((F(*a) - F(*b)) / (2 * h))
    fd = np.array(fd)
    assert np.max(np.abs(got - fd)) <= 1e-6 * np.max(np.abs(fd))


def _bubble(n=16, centre=(0.0, 0.0), radius=0.45):
    return inputs.adjoint_bubble(n, centre=centre, radius=radius)


def test_taped_step_equals_plain_step_and_replay_reproduces_it():
    case = _bubble(24, radius=0.4)
    cfg = case["cfg"]
    base = O.Oracle(cfg).init(case["phi"], case["prim_N"], case["prim_P"])
    base.step_single_dt(2)
    qN, qP, phi = base.state()
    plain, taped, replay = O.Oracle(cfg), O.Oracle(cfg), O.Oracle(cfg)
    for o in (plain, taped, replay):
        o.set_state(qN, qP, phi)
    plain.step_single_dt(1)
    rec = taped.step_taped()
    replay.replay_step(rec)
    for a, b in ((plain, taped), (taped, replay)):
        assert np.array_equal(_state(a), _state(b))
    assert np.array_equal(plain.state()[2], taped.state()[2])
    assert np.array_equal(rec["phi2"], taped.state()[2])
    assert plain.t == taped.t == replay.t


def test_rhs_adjoint_equals_bruteforce_jacobian():
    """Every entry of J_L (both fluids, 8 x 16 x 16 states) by central
    column differences against every row of the transposed map.  The step
    is small (1e-8 of the component's largest magnitude) because small cut
    cells divide by their volume fraction, which makes the map strongly
    curved there."""
    case = _bubble(16, radius=0.4)
    cfg = case["cfg"]
    o = O.Oracle(cfg).init(case["phi"], case["prim_N"], case["prim_P"])
    o.step_single_dt(1)
    qN, qP, phi = o.state()
    Q0 = np.stack([qN, qP])
    lf = O.Oracle(cfg)
    lf.set_state(qN, qP, phi)
    lf4 = lf.step_taped()["lf"][:4]
    n = Q0.size
    scale = (np.abs(Q0).reshape(2, 4, -1).max(axis=2)[:, :, None, None] * np.ones_like(Q0)).ravel()

    def F(q):
        x = O.Oracle(cfg)
        x.set_state(q[0], q[1], phi)
        return x.rhs_frozen(lf4).ravel()

    Jfd = np.empty((n, n))
    for col in range(n):
        e = np.zeros(n)
        e[col] = h = 1e-8 * scale[col]
        Jfd[:, col] = (F((Q0.ravel() + e).reshape(Q0.shape)) -
                       F((Q0.ravel() - e).reshape(Q0.shape))) / (2 * h)
    x = O.Oracle(cfg)
    x.set_state(qN, qP, phi)
    Jad = np.empty((n, n))
    for row in range(n):
        mu = np.zeros(n)
        mu[row] = 1.0
        Jad[row] = x.rhs_adjoint(lf4, mu.reshape(Q0.shape)).ravel()
    rowmax = np.abs(Jfd).max(axis=1, keepdims=True) + 1e-300
    assert np.all(np.abs(Jfd - Jad) <= 1e-5 * rowmax)
    assert np.count_nonzero(Jad) > 10 * n  # the map really couples neighbours


@pytest.mark.parametrize("k", [0, 1])
def test_mix_adjoint_is_the_exact_transpose(k):
    case = _bubble(20, radius=0.37)
    cfg = case["cfg"]
    o = O.Oracle(cfg).init(case["phi"], case["prim_N"], case["prim_P"])
    _, _, phi = o.state()
    rng = np.random.default_rng(k)
    v = rng.normal(size=(2, 4, 20, 20))
    lam = rng.normal(size=(4, 20, 20))
    x = O.Oracle(cfg)
    x.set_state(v[0], v[1], phi)
    x.mix_only(k)
    Mv = _state(x)[k]
    assert not np.allclose(Mv, v[k])  # some cells do mix
    y = O.Oracle(cfg)
    y.set_state(v[0], v[1], phi)
    MTl = y.mix_adjoint(k, lam)
    a, b = np.sum(lam * Mv), np.sum(MTl * v[k])
    assert abs(a - b) <= 1e-12 * (np.sum(np.abs(lam * Mv)) + 1e-300)


def test_adjoint_step_satisfies_conservation_identities():
    """The frozen step conserves each fluid's mass and the two fluids'
    summed momentum and energy for every state (periodic box), so the
    transposed step maps each of these constant adjoints onto itself."""
    case = inputs.periodic_bubble(24)
    cfg = case["cfg"]
    o = O.Oracle(cfg).init(case["phi"], case["prim_N"], case["prim_P"])
    o.step_single_dt(1)
    q = o.state()
    rec = o.step_taped()
    x = O.Oracle(cfg)
    x.set_state(*q)
    shape = (2, 4, cfg["ny"], cfg["nx"])
    seeds = []
    for k in (0, 1):
        lam = np.zeros(shape)
        lam[k, 0] = 1.0
        seeds.append(lam)
    for m in (1, 2, 3):
        lam = np.zeros(shape)
        lam[:, m] = 1.0
        seeds.append(lam)
    for lam in seeds:
        out = x.adjoint_step(rec, lam)
        assert np.max(np.abs(out - lam)) <= 1e-11


def test_wall_pressure_gradient_matches_central_differences():
    """J = sum over the x = 1 wall column of p_water dy after 20 frozen
    steps; its gradient with respect to the initial gas pressure field by
    the adjoint chain (steps, then initialisation) against central
    differences (eps 1e-6) along seeded unit directions on bubble cells."""
    n, N = 32, 20
    case = inputs.adjoint_bubble(n, centre=(0.45, 0.0), radius=0.3)
    cfg = case["cfg"]
    g1, pi1, dy = cfg["gamma"][1], cfg["pinf"][1], cfg["dy"]
    o = O.Oracle(cfg).init(case["phi"], case["prim_N"], case["prim_P"])
    states, recs = [], []
    for _ in range(N):
        states.append(o.state())
        recs.append(o.step_taped())
    qN, qP, phi = o.state()
    a_end = O.Oracle(cfg)
    a_end.set_state(qN, qP, phi)
    aw = a_end.geometry()["alpha"][:, -1]

    def J(qp):
        q = qp[:, :, -1]
        rho, u, v, E = q[0] / aw, q[1] / q[0], q[2] / q[0], q[3] / aw
        return np.sum((g1 - 1) * (E - 0.5 * rho * (u * u + v * v)) - g1 * pi1) * dy

    q = qP[:, :, -1]
    u, v = q[1] / q[0], q[2] / q[0]
    lam = np.zeros((2, 4, n, n))
    lam[1, 0, :, -1] = (g1 - 1) * 0.5 * (u * u + v * v) / aw * dy
    lam[1, 1, :, -1] = -(g1 - 1) * u / aw * dy
    lam[1, 2, :, -1] = -(g1 - 1) * v / aw * dy
    lam[1, 3, :, -1] = (g1 - 1) / aw * dy
    for s in reversed(range(N)):
        x = O.Oracle(cfg)
        x.set_state(*states[s])
        lam = x.adjoint_step(recs[s], lam)
    x = O.Oracle(cfg)
    x.set_state(*states[0])
    grad = x.adjoint_init(case["prim_N"], case["prim_P"], lam)[0, 3]

    def J_replay(p_gas):
        pN = case["prim_N"].copy()
        pN[3] = p_gas
        y = O.Oracle(cfg).init(case["phi"], pN, case["prim_P"])
        for r in recs:
            y.replay_step(r)
        return J(y.state()[1])

    assert J_replay(case["prim_N"][3]) == J(qP)
    rng = np.random.default_rng(0)
    bubble = case["phi"] < 0
    eps = 1e-6
    for _ in range(4):
        d = rng.normal(size=(n, n)) * bubble
        d /= np.linalg.norm(d)
        fd = (J_replay(case["prim_N"][3] + eps * d) - J_replay(case["prim_N"][3] - eps * d)) / (2 * eps)
        ad = np.sum(grad * d)
        assert abs(fd - ad) <= 1e-6 * abs(ad)


def test_adjoint_entry_points_require_rk2():
    case = inputs.shock_tube_1d(40, rk_order=3)
    o = O.Oracle(case["cfg"]).init(case["phi"], case["prim_N"], case["prim_P"])
    with pytest.raises(RuntimeError):
        o.step_taped()
