"""The adjoint of the frozen single-time-step RK2 step on the GPU, through
the C-ABI: recording does not change the steps, the frozen replay
reproduces them bitwise, each adjoint step and the adjoint of the
initialisation equal the oracle's, the gradient of a wall-pressure
functional equals central differences of the replayed forward, and the
checkpointed torch.autograd.Function equals the one-tape result bitwise.

Gradient checks use the gas-water bubble in nondimensional units (states
of order one), where WENO5-JS's absolute epsilon leaves the forward map
smooth on the scale of a difference step."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs

pytestmark = pytest.mark.gpu


def _sif():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_03917_gb300 import sif
    return sif


def _arrays(case):
    return [np.ascontiguousarray(case[x], dtype=np.float64) for x in ("phi", "prim_N", "prim_P")]


def _q(solver):
    qN, qP, _ = solver.state()
    return np.ascontiguousarray(np.stack([qN, qP]))


def _rel(a, b):
    return np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300)


def test_recording_does_not_change_the_steps():
    sif = _sif()
    case = inputs.adjoint_bubble(64, centre=(0.3, 0.1), radius=0.3)
    a = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    b = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    b.tape_reset(6)
    a.step_single_dt(6)
    b.step_single_dt(6)
    assert b.tape_length == 6
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)
    assert a.t == b.t


def test_replay_reproduces_each_recorded_step_bitwise():
    sif = _sif()
    case = inputs.adjoint_bubble(64, centre=(0.3, 0.1), radius=0.3)
    s = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    s.tape_reset(5)
    states = [_q(s)]
    for _ in range(5):
        s.step_single_dt(1)
        states.append(_q(s))
    before = s.save()
    for n in range(5):
        out = s.replay_step(n, states[n])
        assert np.array_equal(out, states[n + 1]), n
    assert s.save() == before  # the context's state is untouched


def _oracle_at(case, nsteps):
    """Oracle advanced nsteps taped steps from the initial data; returns the
    oracle (at step nsteps) and the schedule records."""
    o = O.Oracle(case["cfg"]).init(case["phi"], case["prim_N"], case["prim_P"])
    recs = [o.step_taped() for _ in range(nsteps)]
    return o, recs


def test_adjoint_steps_and_init_match_the_oracle():
    sif = _sif()
    N = 3
    case = inputs.adjoint_bubble(40, centre=(0.3, 0.0), radius=0.35)
    s = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    s.tape_reset(N)
    s.step_single_dt(N)
    rng = np.random.default_rng(11)
    lam0 = rng.normal(size=(2, 4, 40, 40))
    lam_g = lam0.copy()
    lam_o = lam0.copy()
    for n in reversed(range(N)):
        lam_g = s.adjoint_step(n, np.ascontiguousarray(lam_g))
        # the oracle sits at the start of step n with the same history (its
        # stencil states start the extension); step n's record comes from
        # a second run one step longer
        o, _ = _oracle_at(case, n)
        rec_n = _oracle_at(case, n + 1)[1][n]
        lam_o = o.adjoint_step(rec_n, lam_o)
        for k in range(2):
            for m in range(4):
                e = _rel(lam_g[k, m], lam_o[k, m])
                assert e <= 1e-10, (n, k, m, e)
    phi, pN, pP = _arrays(case)
    g_init = s.adjoint_init(phi, pN, pP, np.ascontiguousarray(lam_g))
    o0 = O.Oracle(case["cfg"]).init(case["phi"], case["prim_N"], case["prim_P"])
    o_init = o0.adjoint_init(case["prim_N"], case["prim_P"], lam_o)
    for k in range(2):
        for m in range(4):
            if np.abs(o_init[k, m]).sum() > 0:
                assert _rel(g_init[k, m], o_init[k, m]) <= 1e-10, (k, m)


def _wall_seed(q, cfg):
    """dJ/dq for J = sum_j p_P(nx-1, j) dy with a pure-water wall column."""
    g, pi, dy = cfg["gamma"][1], cfg["pinf"][1], cfg["dy"]
    w = q[1, :, :, -1]
    rho, u, v = w[0], w[1] / w[0], w[2] / w[0]
    lam = np.zeros_like(q)
    lam[1, 0, :, -1] = (g - 1) * 0.5 * (u * u + v * v) * dy
    lam[1, 1, :, -1] = -(g - 1) * u * dy
    lam[1, 2, :, -1] = -(g - 1) * v * dy
    lam[1, 3, :, -1] = (g - 1) * dy
    return lam


def _wall_J(q, cfg):
    g, pi, dy = cfg["gamma"][1], cfg["pinf"][1], cfg["dy"]
    w = q[1, :, :, -1]
    p = (g - 1) * (w[3] - 0.5 * (w[1] ** 2 + w[2] ** 2) / w[0]) - g * pi
    return p.sum() * dy


def _gradient_vs_fd(n, N, centre, radius, ndir, tol):
    """Adjoint gradient of J with respect to the initial gas pressure field
    against central differences (eps 1e-6, fourth order) of the replayed
    forward along seeded unit directions on bubble cells, the difference
    measured against each direction's derivative and against the
    gradient's norm; device buffers throughout."""
    sif = _sif()
    import torch
    case = inputs.adjoint_bubble(n, centre=centre, radius=radius)
    cfg = case["cfg"]
    dev = torch.device("cuda:0")
    phi, pN, pP = (torch.tensor(a, dtype=torch.float64, device=dev) for a in _arrays(case))
    s = sif.Solver(cfg).init_fluids(phi, pN, pP)
    s.tape_reset(N)
    s.step_single_dt(N)
    q = torch.empty((2, 4, n, n), dtype=torch.float64, device=dev)
    phi_end = torch.empty((n, n), dtype=torch.float64, device=dev)
    s.state_into(q[0], q[1], phi_end)
    qh = q.cpu().numpy()
    lam = torch.tensor(_wall_seed(qh, cfg), device=dev)
    for k in reversed(range(N)):
        s.adjoint_step(k, lam, lam)
    gp = torch.empty_like(lam)
    s.adjoint_init(phi, pN, pP, lam, gp)
    grad = gp[0, 3].cpu().numpy()
    aux = sif.Solver(cfg)
    w = torch.empty_like(q)

    def J_of(p_gas):
        pn = pN.clone()
        pn[3] = torch.tensor(p_gas, device=dev)
        aux.init_fluids(phi, pn, pP)
        aux.state_into(w[0], w[1], phi_end)
        for k in range(N):
            s.replay_step(k, w, w)
        return _wall_J(w.cpu().numpy(), cfg)

    p0 = case["prim_N"][3]
    assert J_of(p0) == _wall_J(qh, cfg)
    # the largest directional derivative over unit directions on bubble
    # cells: the scale against which a difference quotient is judged (a
    # direction nearly orthogonal to the gradient has a tiny derivative
    # that rounding over hundreds of steps blurs at the 1e-10 level)
    gnorm = float(np.linalg.norm(grad * (case["phi"] < 0)))
    rng = np.random.default_rng(5)
    bubble = case["phi"] < 0
    eps = 1e-6
    worst = 0.0
    for _ in range(ndir):
        d = rng.normal(size=bubble.shape) * bubble
        d /= np.linalg.norm(d)
        # fourth-order central difference (steps eps and 2 eps): the WENO5
        # weights curve on a scale of about sqrt(weno eps) = 1e-3 in these
        # units, which leaves the second-order difference near 1e-6
        fd = (8.0 * (J_of(p0 + eps * d) - J_of(p0 - eps * d)) -
              (J_of(p0 + 2 * eps * d) - J_of(p0 - 2 * eps * d))) / (12 * eps)
        ad = float(np.sum(grad * d))
        # per direction, relative to that direction's derivative (the bar
        # the check is held to), and relative to the gradient's norm.  The
        # differences of J carry a rounding floor (about 1e-10 absolute
        # after hundreds of replayed steps): a direction whose derivative
        # lies below 1 % of the gradient's norm is judged against 1 % of it
        e_dir = abs(fd - ad) / max(abs(ad), 1e-2 * gnorm)
        e = abs(fd - ad) / gnorm
        worst = max(worst, e_dir)
        assert e_dir <= tol, (fd, ad, gnorm, e_dir)
        assert e <= tol, (fd, ad, gnorm, e)
    return worst


def test_wall_pressure_gradient_matches_central_differences():
    _gradient_vs_fd(96, 40, centre=(0.55, 0.0), radius=0.25, ndir=16, tol=1e-6)


def test_wall_pressure_gradient_512_bubble_200_steps():
    """The gas-water bubble at 512 x 512 after 200 steps, bubble centred at
    x = 0.7 so that its signal reaches the x = 1 wall within the run."""
    _gradient_vs_fd(512, 200, centre=(0.7, 0.0), radius=0.12, ndir=16, tol=1e-6)


def test_checkpointed_autograd_equals_one_tape_and_manual_chain():
    sif = _sif()
    import torch
    from paper_1905_03917_gb300 import adjoint
    case = inputs.adjoint_bubble(80, centre=(0.5, 0.0), radius=0.25)
    cfg = case["cfg"]
    dev = torch.device("cuda:0")
    phi = torch.tensor(case["phi"], dtype=torch.float64, device=dev)
    pP = torch.tensor(case["prim_P"], dtype=torch.float64, device=dev)
    grads = []
    for every in (7, 30):
        pN = torch.tensor(case["prim_N"], dtype=torch.float64, device=dev, requires_grad=True)
        s = sif.Solver(cfg)
        q, _ = adjoint.frozen_steps(s, phi, pN, pP, nsteps=30, every=every)
        J = adjoint.wall_pressure(q, cfg)
        J.backward()
        grads.append(pN.grad.detach().cpu().numpy())
    assert np.array_equal(grads[0], grads[1])
    # the same chain by hand
    s = sif.Solver(cfg).init_fluids(*_arrays(case))
    s.tape_reset(30)
    s.step_single_dt(30)
    lam = _wall_seed(_q(s), cfg)
    for k in reversed(range(30)):
        lam = s.adjoint_step(k, lam)
    phi_h, pN_h, pP_h = _arrays(case)
    g = s.adjoint_init(phi_h, pN_h, pP_h, lam)[0]
    assert np.allclose(grads[0], g, rtol=1e-12, atol=1e-300 + 1e-14 * np.abs(g).max())
    assert np.abs(grads[0][3]).max() > 0


def test_tape_errors_are_reported():
    sif = _sif()
    case = inputs.adjoint_bubble(32, radius=0.3)
    s = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    s.tape_reset(2)
    s.step_single_dt(2)
    with pytest.raises(sif.SifError) as e:
        s.step_single_dt(1)
    assert e.value.code == sif.EINVAL
    with pytest.raises(sif.SifError) as e:
        s.step_multi_dt(1)
    assert e.value.code == sif.ESTATE
    with pytest.raises(sif.SifError) as e:
        s.adjoint_step(2, np.zeros((2, 4, 32, 32)))
    assert e.value.code == sif.EINVAL
    s.tape_reset(0)
    s.step_multi_dt(1)  # recording off again
    tube = inputs.shock_tube_1d(64, rk_order=3)
    r = sif.Solver(tube["cfg"]).init_fluids(*_arrays(tube))
    with pytest.raises(sif.SifError) as e:
        r.tape_reset(4)
    assert e.value.code == sif.EINVAL
