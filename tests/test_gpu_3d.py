"""Parity of the three-dimensional CUDA path (include/sif3d.h, through the
C-ABI) with the 3D oracle on seeded inputs: the cube's cut-cell geometry to
round-off, one single step and one accelerated cycle (Sec. 3.1) to 1e-12
relative L1 per fluid and component, 20 cycles to 1e-8, the sub-step counts
cycle by cycle, conservation with the Eq. 8-9 correction, the bitwise
ratio-one reduction, and the 128^3 droplet of Table 1's 3D row in the
bench's launch configuration."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _sif():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_03917_gb300 import sif
    return sif


def rel_l1(a, b, floor):
    return np.abs(a - b).sum() / max(np.abs(b).sum(), floor)


def sound_scale(case):
    cfg = case["cfg"]
    c = 0.0
    for k, pr in ((0, case["prim_N"]), (1, case["prim_P"])):
        c = max(c, float(np.sqrt(cfg["gamma"][k] * (pr[4] + cfg["pinf"][k]) / pr[0]).max()))
    return c


def compare3(gs, os_, tol, cref):
    """The 2D tests' measure with five components: relative L1 per fluid and
    component (momentum against mass x the largest initial sound speed
    where the momentum is smaller) and the largest element-wise difference
    relative to the component's scale (tol, ten times tol for long runs)."""
    worst = 0.0
    tol_max = tol if tol < 1e-10 else 10.0 * tol
    for k in range(2):
        mass = np.abs(os_[k][0]).sum()
        rho_max = np.abs(os_[k][0]).max()
        for m in range(5):
            mom = m in (1, 2, 3)
            floor = max(mass * cref, 1e-300) if mom else 1e-300
            e = rel_l1(gs[k][m], os_[k][m], floor)
            assert e <= tol, (k, m, e)
            scale = np.abs(os_[k][m]).max()
            if mom:
                scale = max(scale, rho_max * cref)
            if scale > 0.0:
                e_max = np.abs(gs[k][m] - os_[k][m]).max() / scale
                assert e_max <= tol_max, ("max", k, m, e_max)
                worst = max(worst, e_max)
            worst = max(worst, e)
    e = rel_l1(gs[2], os_[2], 1e-300)
    assert e <= tol, ("phi", e)
    return max(worst, e)


def pair(case, **kw):
    sif = _sif()
    cfg = dict(case["cfg"], **kw)
    arrs = [np.ascontiguousarray(case[x], dtype=np.float64) for x in ("phi", "prim_N", "prim_P")]
    g = sif.Solver3(cfg).init_fluids(*arrs)
    o = O.Oracle3(cfg).init(*arrs)
    return g, o


def pulse_droplet(n=16):
    c = I.droplet_translation_3d(n)
    X, Y, Z = I._centres3(c["cfg"])
    r2 = (X - 0.25) ** 2 + (Y - 0.3) ** 2 + (Z - 0.7) ** 2
    c["prim_P"][4] = 1.0 + 0.3 * np.exp(-r2 / 0.01)
    return c


def gas_bubble(n=16):
    """A high-pressure stiffened-gas bubble off-centre in water, reflective
    walls: a violent 3D case with a moving, deforming interface."""
    water = {"gamma": 4.4, "pinf": 6.0e8}
    cfg = I.config3(n, n, n, 1.0 / n, I.AIR, water, ["reflect"] * 6)
    X, Y, Z = I._centres3(cfg)
    phi = np.sqrt((X - 0.45) ** 2 + (Y - 0.52) ** 2 + (Z - 0.48) ** 2) - 0.22
    pN = I._uniform3(X.shape, 1.0, 0.0, 0.0, 0.0, 1.0e8)
    pP = I._uniform3(X.shape, 1000.0, 0.0, 0.0, 0.0, 1.0e5)
    return {"name": "gas_bubble_3d", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


CASES = {
    "shock_bubble": lambda: I.shock_bubble_3d(8),
    "droplet": lambda: pulse_droplet(16),
    "gas_bubble": lambda: gas_bubble(16),
}


def test_geometry_matches_oracle():
    c = I.shock_bubble_3d(12, seed=3, perturb=0.1)
    g, o = pair(c)
    gg, og = g.geometry(), o.geometry()
    for k in ("alpha", "ax", "ay", "az", "sx", "sy", "sz"):
        assert np.abs(gg[k] - og[k]).max() <= 1e-14, k


@pytest.mark.parametrize("name", sorted(CASES))
def test_single_step_matches_oracle(name):
    c = CASES[name]()
    g, o = pair(c)
    cref = sound_scale(c)
    for _ in range(2):
        gi = g.step_single_dt(1)
        oi = o.step_single_dt(1)
        assert gi["t"] == pytest.approx(oi["t"], rel=1e-12)
        assert gi["open_updates"] == oi["open_updates"]
        compare3(g.state(), o.state(), 1e-12, cref)


@pytest.mark.parametrize("name", sorted(CASES))
def test_cycle_matches_oracle(name):
    c = CASES[name]()
    g, o = pair(c)
    cref = sound_scale(c)
    gi = g.step_multi_dt(1)
    oi = o.step_multi_dt(1)
    assert gi["substeps"] == oi["substeps"] and gi["role_fluid1"] == oi["role_fluid1"]
    assert gi["t"] == pytest.approx(oi["t"], rel=1e-12)
    assert gi["open_updates"] == oi["open_updates"]
    compare3(g.state(), o.state(), 1e-12, cref)


def test_twenty_cycles_match_oracle():
    c = pulse_droplet(16)
    g, o = pair(c)
    cref = sound_scale(c)
    for _ in range(20):
        gi = g.step_multi_dt(1)
        oi = o.step_multi_dt(1)
        assert gi["substeps"] == oi["substeps"]
    assert g.t == pytest.approx(o.t, rel=1e-10)
    compare3(g.state(), o.state(), 1e-8, cref)


def test_hundred_cycles_match_oracle():
    """The long-run bar: 100 accelerated cycles (about 350 water sub-steps)
    of the droplet with its pressure pulse to 1e-8."""
    c = pulse_droplet(16)
    g, o = pair(c)
    for _ in range(100):
        gi, oi = g.step_multi_dt(1), o.step_multi_dt(1)
        assert gi["substeps"] == oi["substeps"]
    assert g.t == pytest.approx(o.t, rel=1e-10)
    compare3(g.state(), o.state(), 1e-8, sound_scale(c))


def test_conservation_with_correction_on_gpu():
    c = pulse_droplet(16)
    g, _ = pair(c)
    i0 = g.integrals()
    info = g.step_multi_dt(3)
    assert info["substeps"] >= 3
    i1 = g.integrals()
    assert np.all(np.abs(i1[:, 0] - i0[:, 0]) <= 1e-13 * np.abs(i0[:, 0]))
    tot0, tot1 = i0.sum(axis=0), i1.sum(axis=0)
    assert abs(tot1[4] - tot0[4]) <= 1e-13 * abs(tot0[4])
    scale = np.abs(i0[:, 1]).sum()
    assert np.all(np.abs(tot1[1:4] - tot0[1:4]) <= 1e-13 * scale)


def test_ratio_one_cycle_is_the_single_step_bitwise_on_gpu():
    c = pulse_droplet(12)
    sif = _sif()
    arrs = [np.ascontiguousarray(c[x]) for x in ("phi", "prim_N", "prim_P")]
    a = sif.Solver3(dict(c["cfg"], force_ratio_one=1)).init_fluids(*arrs)
    b = sif.Solver3(c["cfg"]).init_fluids(*arrs)
    a.step_multi_dt(2)
    b.step_single_dt(2)
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)


def test_device_tensors_and_host_arrays_agree():
    torch = pytest.importorskip("torch")
    sif = _sif()
    c = pulse_droplet(12)
    arrs = [np.ascontiguousarray(c[x]) for x in ("phi", "prim_N", "prim_P")]
    a = sif.Solver3(c["cfg"]).init_fluids(*arrs)
    b = sif.Solver3(c["cfg"]).init_fluids(*(torch.from_numpy(x).cuda() for x in arrs))
    a.step_multi_dt(1)
    b.step_multi_dt(1)
    out = [torch.empty(s, dtype=torch.float64, device="cuda")
           for s in ((5,) + a.shape, (5,) + a.shape, a.shape)]
    b.state_into(*out)
    torch.cuda.synchronize()
    for x, y in zip(a.state(), out):
        assert np.array_equal(x, y.cpu().numpy())


def test_droplet_128_one_cycle_matches_oracle():
    """Table 1's 3D row at its full size, one accelerated cycle in the
    bench's launch configuration (one call per cycle)."""
    c = I.droplet_translation_3d(128)
    g, o = pair(c)
    gi = g.step_multi_dt(1)
    oi = o.step_multi_dt(1)
    assert gi["substeps"] == oi["substeps"] and gi["role_fluid1"] == oi["role_fluid1"]
    assert gi["open_updates"] == oi["open_updates"]
    compare3(g.state(), o.state(), 1e-12, sound_scale(c))


# -- surface tension (Eq. 10) ---------------------------------------------------

def test_surface_tension_matches_oracle():
    # a gas sphere out of equilibrium (the jump drives its motion)
    c = I.static_drop_3d(16, equilibrium=False)
    g, o = pair(c)
    cref = sound_scale(c)
    for _ in range(2):
        g.step_single_dt(1)
        o.step_single_dt(1)
        compare3(g.state(), o.state(), 1e-12, cref)
    gi, oi = g.step_multi_dt(1), o.step_multi_dt(1)
    assert gi["substeps"] == oi["substeps"]
    compare3(g.state(), o.state(), 1e-12, cref)


def test_static_sphere_keeps_the_laplace_jump_on_gpu():
    """Laplace's law for a sphere, 2 sigma / R = 288, held by the CUDA path
    within 2 % over 60 steps on 24^3 (closed form)."""
    c = I.static_drop_3d(24)
    sif = _sif()
    s = sif.Solver3(c["cfg"]).init_fluids(*(np.ascontiguousarray(c[x])
                                            for x in ("phi", "prim_N", "prim_P")))
    X, Y, Z = I._centres3(c["cfg"])
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    d = 1.0 / 24
    for _ in range(6):
        s.step_single_dt(10)
        qN, qP, _ = s.state()
        a = s.geometry()["alpha"]
        inn, out = (r < 0.25 - 2 * d) & (a < 1e-3), (r > 0.25 + 2 * d) & (a > 0.999)

        def pres(q, al, m):
            rho = q[0][m] / al[m]
            u, v, w = (q[x][m] / q[0][m] for x in (1, 2, 3))
            return (0.4 * (q[4][m] / al[m] - 0.5 * rho * (u * u + v * v + w * w))).mean()
        jump = pres(qN, 1 - a, inn) - pres(qP, a, out)
        assert abs(jump / 288.0 - 1.0) <= 0.02, jump


# -- viscosity (Eq. 3, 5) -------------------------------------------------------

def viscous_bubble(n=16):
    """The shock-bubble with both fluids viscous and a shear flow through
    the box: face viscous fluxes in all three directions, the interface
    traction, the viscous time-step limit."""
    c = I.shock_bubble_3d(n // 2)
    c["cfg"]["mu"] = [0.01, 0.005]
    X, Y, Z = I._centres3(c["cfg"])
    for key in ("prim_N", "prim_P"):
        c[key][3] = 0.3 * np.sin(2.0 * np.pi * Y) * np.cos(2.0 * np.pi * X)
    return c


def test_viscosity_matches_oracle():
    c = viscous_bubble(16)
    g, o = pair(c)
    cref = sound_scale(c)
    for _ in range(2):
        gi, oi = g.step_single_dt(1), o.step_single_dt(1)
        assert gi["t"] == pytest.approx(oi["t"], rel=1e-12)
        compare3(g.state(), o.state(), 1e-12, cref)
    gi, oi = g.step_multi_dt(1), o.step_multi_dt(1)
    assert gi["substeps"] == oi["substeps"]
    compare3(g.state(), o.state(), 1e-12, cref)


def test_shear_wave_along_z_decays_at_the_viscous_rate_on_gpu():
    """u = a sin(2 pi z) decays as exp(-nu (2 pi)^2 t) in the CUDA path
    (closed form)."""
    import math
    n, mu, amp = 32, 0.01, 0.01
    cfg = I.config3(4, 4, n, 1.0 / n, I.AIR, I.AIR, ["periodic"] * 6, mu=[mu, mu])
    X, Y, Z = I._centres3(cfg)
    phi = np.ones_like(X)
    prim = I._uniform3(X.shape, 1.0, 0.0, 0.0, 0.0, 100.0)
    prim[1] = amp * np.sin(2.0 * math.pi * Z)
    s = _sif().Solver3(cfg).init_fluids(phi, prim, prim.copy())
    T = 0.5
    s.step_single_dt(100000, t_end=T)
    qP = s.state()[1]
    u = qP[1] / qP[0]
    a = 2.0 * (u[:, 0, 0] * np.sin(2.0 * math.pi * Z[:, 0, 0])).mean()
    assert a == pytest.approx(amp * math.exp(-mu * (2.0 * math.pi) ** 2 * T), rel=2e-3)


def test_circle_recovery_3d_matches_oracle():
    """Table 3's 3D case (Tait fluids, surface tension, viscosity) at 32^3:
    two single steps and one accelerated cycle against the oracle."""
    c = I.circle_recovery_3d(32)
    g, o = pair(c)
    cref = sound_scale(c)
    for _ in range(2):
        g.step_single_dt(1)
        o.step_single_dt(1)
    compare3(g.state(), o.state(), 1e-12, cref)
    gi, oi = g.step_multi_dt(1), o.step_multi_dt(1)
    assert gi["substeps"] == oi["substeps"] and gi["role_fluid1"] == oi["role_fluid1"]
    compare3(g.state(), o.state(), 1e-12, cref)


def test_filament_3d_matches_oracle():
    """Table 4's 3D case (Tait fluids, surface tension, viscosity, SI
    units, symmetry planes) at 16 x 16 x 32."""
    c = I.filament_3d(16)
    g, o = pair(c)
    cref = sound_scale(c)
    for _ in range(2):
        g.step_single_dt(1)
        o.step_single_dt(1)
    compare3(g.state(), o.state(), 1e-12, cref)
    gi, oi = g.step_multi_dt(1), o.step_multi_dt(1)
    assert gi["substeps"] == oi["substeps"] and gi["role_fluid1"] == oi["role_fluid1"]
    compare3(g.state(), o.state(), 1e-12, cref)


# -- error paths of the bounded loops (no fault: host-set limits) -------------

def test_substep_limit_gives_timeout_and_the_context_recovers():
    sif = _sif()
    c = pulse_droplet(16)
    s = sif.Solver3(c["cfg"]).init_fluids(*(np.ascontiguousarray(c[x])
                                            for x in ("phi", "prim_N", "prim_P")))
    saved = s.state()
    s.set_limits(max_substeps=2)
    with pytest.raises(sif.SifError) as e:
        s.step_multi_dt(1)
    assert e.value.code == sif.ETIMEOUT
    s.set_limits(max_substeps=4096)
    s.set_state(*saved)
    assert s.step_multi_dt(1)["substeps"] >= 3


def test_newton_limit_gives_noconv_and_the_context_recovers():
    sif = _sif()
    c = gas_bubble(16)
    s = sif.Solver3(c["cfg"]).init_fluids(*(np.ascontiguousarray(c[x])
                                            for x in ("phi", "prim_N", "prim_P")))
    saved = s.state()
    s.set_limits(newton_iters=1)
    with pytest.raises(sif.SifError) as e:
        s.step_single_dt(1)
    assert e.value.code == sif.ENOCONV
    s.set_limits(newton_iters=50)
    s.set_state(*saved)
    s.step_single_dt(1)


def ragged_case():
    """A grid that fills no brick (8 x 8 x 4) evenly along any axis, with a
    gas bubble off-centre in water and zero-gradient, reflective and
    periodic sides: the bricks' ragged tails."""
    water = {"gamma": 4.4, "pinf": 6.0e8}
    d = 1.0 / 19
    cfg = I.config3(19, 13, 11, d, I.AIR, water,
                    ["zerograd", "zerograd", "reflect", "reflect", "periodic", "periodic"])
    X, Y, Z = I._centres3(cfg)
    phi = np.sqrt((X - 0.55) ** 2 + (Y - 0.33) ** 2 + (Z - 0.3) ** 2) - 0.2
    pN = I._uniform3(X.shape, 1.0, 0.0, 0.0, 0.0, 5.0e7)
    pP = I._uniform3(X.shape, 1000.0, 20.0, 0.0, 0.0, 1.0e5)
    return {"name": "ragged_3d", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


def test_ragged_grid_matches_oracle():
    c = ragged_case()
    g, o = pair(c)
    cref = sound_scale(c)
    gg, og = g.geometry(), o.geometry()
    for k in ("alpha", "ax", "ay", "az", "sx", "sy", "sz"):
        assert np.abs(gg[k] - og[k]).max() <= 1e-14, k
    for _ in range(2):
        gi, oi = g.step_single_dt(1), o.step_single_dt(1)
        assert gi["open_updates"] == oi["open_updates"]
    compare3(g.state(), o.state(), 1e-12, cref)
    for _ in range(3):
        gi, oi = g.step_multi_dt(1), o.step_multi_dt(1)
        assert gi["substeps"] == oi["substeps"]
    compare3(g.state(), o.state(), 1e-11, cref)
