"""Pins of the three-dimensional oracle (oracle/sif_oracle3d.c) against what
geometry, the two-dimensional oracle and conservation fix.

- Cut-cell geometry (Sec. 2.1 with a third pair of faces): exact half-space
  volumes and cut areas of random planes (closed form of a cube cut by a
  plane), the 2D polygon area for a level set constant along z, sphere
  volume and area convergence.
- The step (Eq. 2 in 3D, Eq. 6, Sec. 2.2-2.3): on a 2D case repeated along
  z the 3D single step reproduces the 2D oracle's; a planar tube along each
  axis reproduces the 1D oracle's; permuting the axes permutes the result.
- The accelerated cycle (Sec. 3.1, Eq. 7-9): exact conservation with the
  correction and its loss without it; with dt1 = dt2 forced the cycle is the
  single step bitwise; uniform flow past the droplet keeps its velocity.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs as I


def _below(a, t):
    """Volume of {xi in [0,1]^3 : a . xi <= t} for a > 0 componentwise, and
    its derivative in t (inclusion-exclusion over the cube's vertices)."""
    v = dv = 0.0
    for c in itertools.product((0, 1), repeat=3):
        r = t - sum(ai * ci for ai, ci in zip(a, c))
        if r > 0:
            sg = (-1) ** sum(c)
            v += sg * r ** 3
            dv += sg * r ** 2
    pa = a[0] * a[1] * a[2]
    return v / (6 * pa), dv / (2 * pa)


def _plane_exact(a, b):
    """alpha and S (unit-face areas, pointing into phi >= 0) of phi = a . xi + b."""
    ap = [abs(x) for x in a]
    # reflect each axis with a negative coefficient: xi_d -> 1 - xi_d
    bp = b + sum(x for x in a if x < 0)
    below, dvdt = _below(ap, -bp)
    return 1.0 - below, np.array([x * dvdt for x in a])


def test_plane_volume_and_cut_area_exact():
    rng = np.random.default_rng(3)
    n = 0
    while n < 300:
        a = rng.uniform(-1, 1, 3)
        if min(abs(a)) < 0.05:
            continue
        # a . xi ranges over [sum of negative a_d, sum of positive a_d]
        b = -rng.uniform(np.minimum(a, 0).sum(), np.maximum(a, 0).sum())
        corners = np.array([a[0] * i + a[1] * j + a[2] * k + b
                            for k in (0, 1) for j in (0, 1) for i in (0, 1)])
        al, s = O.cell_alpha3(corners)
        ex, sx = _plane_exact(a, b)
        assert abs(al - ex) <= 1e-12, (a, b, al, ex)
        assert np.abs(s - sx).max() <= 1e-12, (a, b, s, sx)
        n += 1


def test_axis_aligned_plane_cases():
    # a plane phi = x - 0.3: alpha 0.7, S = (-1, 0, 0) ... into P is +x
    c = np.array([i - 0.3 for k in (0, 1) for j in (0, 1) for i in (0, 1)], float)
    al, s = O.cell_alpha3(c)
    assert al == pytest.approx(0.7, abs=1e-15)
    assert np.allclose(s, [1.0, 0.0, 0.0], atol=1e-15)
    assert O.cell_alpha3(np.ones(8))[0] == 1.0 and O.cell_alpha3(-np.ones(8))[0] == 0.0


def test_z_invariant_cell_is_the_2d_polygon():
    rng = np.random.default_rng(5)
    n = 0
    while n < 300:
        c2 = rng.uniform(-1, 1, 4)  # c00, c10, c11, c01
        pos = c2 >= 0
        changes = sum(pos[e] != pos[(e + 1) % 4] for e in range(4))
        if changes == 4:
            continue  # the saddle's two triangles have no single planar patch
        c00, c10, c11, c01 = c2
        corners = np.array([c00, c10, c01, c11] * 2)  # index i + 2 j (+ 4 k)
        al, s = O.cell_alpha3(corners)
        assert al == pytest.approx(O.cell_alpha(*c2), abs=1e-14)
        ef = O.edge_fraction
        sx = ef(c10, c11) - ef(c00, c01)
        sy = ef(c01, c11) - ef(c00, c10)
        assert np.allclose(s, [sx, sy, 0.0], atol=1e-15)
        n += 1


def _sphere_case(n, R=0.3, centre=(0.51, 0.49, 0.5)):
    cfg = I.config3(n, n, n, 1.0 / n, I.AIR, I.HELIUM, ["reflect"] * 6)
    X, Y, Z = I._centres3(cfg)
    phi = R - np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
    sh = phi.shape
    prim = I._uniform3(sh, 1.0, 0.0, 0.0, 0.0, 1.0)
    return cfg, phi, prim


def test_sphere_volume_and_area_converge():
    R = 0.3
    errs_v, errs_a = [], []
    for n in (12, 24):
        cfg, phi, prim = _sphere_case(n, R)
        o = O.Oracle3(cfg).init(phi, prim, prim)
        g = o.geometry()
        dv = cfg["dx"] ** 3
        vol = g["alpha"].sum() * dv
        area = np.sqrt(g["sx"] ** 2 + g["sy"] ** 2 + g["sz"] ** 2).sum()
        errs_v.append(abs(vol - 4.0 / 3.0 * math.pi * R ** 3) / (4.0 / 3.0 * math.pi * R ** 3))
        errs_a.append(abs(area - 4.0 * math.pi * R ** 2) / (4.0 * math.pi * R ** 2))
        # the closed faces sum to zero: S over the whole sphere cancels
        assert abs(g["sx"].sum()) < 1e-12 and abs(g["sz"].sum()) < 1e-12
    # second order in both (the corner means of a curved distance function
    # shift the surface by about h^2 / (4 R), the planar patches cut chords)
    assert errs_v[1] < 0.03 and errs_v[0] / errs_v[1] > 3.5, errs_v
    assert errs_a[1] < 0.02 and errs_a[0] / errs_a[1] > 3.5, errs_a


def _fixed_steps(o, dts, single=True):
    """Single steps of the given sizes: t_end truncates the CFL step."""
    t = o.t
    for dt in dts:
        t = t + dt
        info = o.step_single_dt(1, t_end=t)
        assert info["err"] == 0
    return o


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_step_on_z_invariant_case_is_the_2d_step():
    c2 = I.shock_bubble(48, 12)
    c3 = I.extrude(c2, 4)
    o2 = O.Oracle(c2["cfg"]).init(c2["phi"], c2["prim_N"], c2["prim_P"])
    o3 = O.Oracle3(c3["cfg"]).init(c3["phi"], c3["prim_N"], c3["prim_P"])
    dts = [1.5e-3, 2e-3, 1e-3]  # below both CFL steps (the 3D one has a z term)
    _fixed_steps(o2, dts)
    _fixed_steps(o3, dts)
    q2 = o2.state()
    q3 = o3.state()
    for f in range(2):
        assert np.all(q3[f][3] == 0.0)  # no z momentum appears
        for z in range(4):
            for m2, m3 in ((0, 0), (1, 1), (2, 2), (3, 4)):
                assert _rel(q3[f][m3][z], q2[f][m2]) < 1e-12, (f, m2, z)
    for z in range(4):
        assert _rel(q3[2][z], q2[2]) < 1e-12


def _tube3(case1, axis, nperp=3):
    """The 1D case laid along `axis` of a 3D box nperp cells wide across it
    (periodic across), velocity along the axis."""
    c1 = case1["cfg"]
    n = c1["nx"]
    mats = [{"gamma": c1["gamma"][k], "pinf": c1["pinf"][k]} for k in range(2)]
    for k in range(2):
        if c1.get("tait") and c1["tait"][k] is not None:
            mats[k]["tait"] = tuple(c1["tait"][k])
    dims = [nperp, nperp, nperp]
    dims[axis] = n
    bc = ["periodic"] * 6
    bc[2 * axis], bc[2 * axis + 1] = c1["bc"][0], c1["bc"][1]
    cfg = I.config3(dims[0], dims[1], dims[2], c1["dx"], mats[0], mats[1], bc,
                    **{k: c1[k] for k in ("cfl", "band", "ext_iters", "reinit_iters")})
    shape = (dims[2], dims[1], dims[0])
    line = [1, 1, 1]
    line[2 - axis] = n

    def lay(v):
        return np.broadcast_to(np.asarray(v).reshape(line), shape).copy()

    def prim(p1):
        out = np.zeros((5,) + shape)
        out[0], out[1 + axis], out[4] = lay(p1[0, 0]), lay(p1[1, 0]), lay(p1[3, 0])
        return out

    return cfg, lay(case1["phi"][0]), prim(case1["prim_N"]), prim(case1["prim_P"])


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_planar_tube_along_each_axis_is_the_1d_step(axis):
    c1 = I.gas_water_tube(60)
    o1 = O.Oracle(c1["cfg"]).init(c1["phi"], c1["prim_N"], c1["prim_P"])
    cfg, phi, pN, pP = _tube3(c1, axis)
    o3 = O.Oracle3(cfg).init(phi, pN, pP)
    dts = [3.0e-6] * 6  # below both CFL steps
    _fixed_steps(o1, dts)
    _fixed_steps(o3, dts)
    q1 = o1.state()
    q3 = o3.state()
    take = [slice(0, 1)] * 3
    take[2 - axis] = slice(None)
    for f in range(2):
        for m1, m3 in ((0, 0), (1, 1 + axis), (3, 4)):
            got = q3[f][m3][tuple(take)].ravel()
            assert _rel(got, q1[f][m1][0]) < 1e-12, (f, m1)
        for other in range(3):
            if other != axis:
                assert np.all(q3[f][1 + other] == 0.0)
    assert _rel(q3[2][tuple(take)].ravel(), q1[2][0]) < 1e-12


def _permute_case(case):
    """x -> y -> z -> x: the box, boundaries, level set and velocities
    rotated so that old axis d becomes new axis d + 1 (mod 3)."""
    cfg = dict(case["cfg"])
    cfg["nx"], cfg["ny"], cfg["nz"] = case["cfg"]["nz"], case["cfg"]["nx"], case["cfg"]["ny"]
    bc = case["cfg"]["bc"]
    cfg["bc"] = [bc[4], bc[5], bc[0], bc[1], bc[2], bc[3]]

    def arr(a):  # (z, y, x) -> (y', x', ... ) with x' = old z, y' = old x, z' = old y
        return np.ascontiguousarray(np.transpose(a, (1, 2, 0)))

    def prim(p):
        return np.stack([arr(p[0]), arr(p[3]), arr(p[1]), arr(p[2]), arr(p[4])])

    return {"cfg": cfg, "phi": arr(case["phi"]), "prim_N": prim(case["prim_N"]),
            "prim_P": prim(case["prim_P"])}


def test_permuted_axes_give_the_permuted_result():
    c = I.shock_bubble_3d(8)
    cp = _permute_case(c)
    oa = O.Oracle3(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    ob = O.Oracle3(cp["cfg"]).init(cp["phi"], cp["prim_N"], cp["prim_P"])
    for o in (oa, ob):
        o.step_single_dt(2)
        o.step_multi_dt(1)
    assert oa.t == pytest.approx(ob.t, rel=1e-13)
    qa, qb = oa.state(), ob.state()
    back = _permute_case({"cfg": c["cfg"], "phi": qa[2], "prim_N": qa[0], "prim_P": qa[1]})
    for f, key in ((0, "prim_N"), (1, "prim_P")):
        for m in range(5):
            assert _rel(qb[f][m], back[key][m]) < 1e-11, (f, m)
    assert _rel(qb[2], back["phi"]) < 1e-11


def _pulse_droplet(n=16):
    c = I.droplet_translation_3d(n)
    X, Y, Z = I._centres3(c["cfg"])
    r2 = (X - 0.25) ** 2 + (Y - 0.3) ** 2 + (Z - 0.7) ** 2
    c["prim_P"][4] = 1.0 + 0.3 * np.exp(-r2 / 0.01)
    return c


def test_cycle_conserves_with_correction_only():
    c = _pulse_droplet()
    drift = {}
    for corr in (1, 0):
        cfg = dict(c["cfg"], flux_correction=corr)
        o = O.Oracle3(cfg).init(c["phi"], c["prim_N"], c["prim_P"])
        i0 = o.integrals()
        info = o.step_multi_dt(2)
        assert info["err"] == 0 and info["substeps"] >= 3
        i1 = o.integrals()
        tot0, tot1 = i0.sum(axis=0), i1.sum(axis=0)
        assert abs(i1[0, 0] - i0[0, 0]) <= 1e-13 * i0[0, 0]
        assert abs(i1[1, 0] - i0[1, 0]) <= 1e-13 * i0[1, 0]
        drift[corr] = abs(tot1[4] - tot0[4]) / tot0[4]
        scale = np.abs(i0[:, 1]).sum()
        if corr:
            assert np.all(np.abs(tot1[1:4] - tot0[1:4]) <= 1e-13 * scale)
    assert drift[1] <= 1e-14 and drift[0] > 1e3 * max(drift[1], 1e-17), drift


def test_ratio_one_cycle_is_the_single_step_bitwise():
    c = _pulse_droplet(12)
    oa = O.Oracle3(dict(c["cfg"], force_ratio_one=1)).init(c["phi"], c["prim_N"], c["prim_P"])
    ob = O.Oracle3(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    oa.step_multi_dt(2)
    ob.step_single_dt(2)
    for a, b in zip(oa.state(), ob.state()):
        assert np.array_equal(a, b)


def test_uniform_flow_keeps_each_fluids_mean_velocity():
    """Both fluids at one pressure moving with one velocity: the interface
    exchange (p_I S, which cancels over the closed droplet surface at a
    uniform p_I) leaves each fluid's momentum / mass at u, and nothing
    creates transverse momentum (cut cells' own velocities are not exact:
    extension and mixing of slivers perturb them)."""
    c = I.droplet_translation_3d(16)
    u0 = c["prim_N"][1].flat[0]
    o = O.Oracle3(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    info = o.step_multi_dt(3)
    assert info["err"] == 0 and info["substeps"] >= 3
    it = o.integrals()
    for f in range(2):
        assert abs(it[f, 1] / it[f, 0] / u0 - 1.0) < 1e-4
        assert np.abs(it[f, 2:4]).max() <= 1e-14 * abs(it[f, 1])


# -- surface tension (Eq. 10) in 3D: Laplace's law for a sphere ---------------

def _sphere_curvature_error(n):
    c = I.static_drop_3d(n)
    o = O.Oracle3(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    g = o.geometry()
    X, Y, Z = I._centres3(c["cfg"])
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    cut = (g["sx"] != 0) | (g["sy"] != 0) | (g["sz"] != 0)
    err = max(abs(o.curvature(i, j, k) - 2.0 / r[k, j, i]) for k, j, i in zip(*np.nonzero(cut)))
    return err * 0.25 / 2.0  # relative to 2 / R


def test_curvature_of_spheres_converges_second_order():
    # phi = r - R: every level set is a sphere, of mean curvature 2 / r
    e16, e32 = _sphere_curvature_error(16), _sphere_curvature_error(32)
    assert e32 < 5e-3 and np.log2(e16 / e32) >= 1.8, (e16, e32)


def test_curvature_of_a_cylinder_is_the_2d_curvature():
    c2 = I.static_drop(32, liquid=False)
    c3 = I.extrude(c2, 4)
    c3["cfg"]["sigma"] = c2["cfg"]["sigma"]
    o2 = O.Oracle(c2["cfg"]).init(c2["phi"], c2["prim_N"], c2["prim_P"])
    o3 = O.Oracle3(c3["cfg"]).init(c3["phi"], c3["prim_N"], c3["prim_P"])
    for i, j in ((12, 16), (16, 12), (13, 13), (19, 20)):
        assert o3.curvature(i, j, 2) == pytest.approx(o2.curvature(i, j), rel=1e-12, abs=1e-12)


def test_curvature_of_a_plane_is_zero():
    cfg = I.config3(12, 12, 12, 1.0 / 12, I.AIR, I.HELIUM, ["reflect"] * 6, sigma=1.0)
    X, Y, Z = I._centres3(cfg)
    phi = 0.3 * X - 0.5 * Y + 0.81 * Z - 0.4
    prim = I._uniform3(phi.shape, 1.0, 0.0, 0.0, 0.0, 1.0)
    o = O.Oracle3(cfg).init(phi, prim, prim)
    assert max(abs(o.curvature(i, j, k)) for i in range(1, 11) for j in range(1, 11)
               for k in range(1, 11)) <= 1e-9


def _laplace_jump_3d(n, steps, sigma=36.0, equilibrium=True, multi=False):
    c = I.static_drop_3d(n, sigma=sigma, equilibrium=equilibrium)
    o = O.Oracle3(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    X, Y, Z = I._centres3(c["cfg"])
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    d = 1.0 / n
    I0 = o.integrals()
    hist = []
    for s in range(steps):
        (o.step_multi_dt if multi else o.step_single_dt)(1)
        if s % 10 == 9:
            qN, qP, _ = o.state()
            a = o.geometry()["alpha"]
            inn, out = (r < 0.25 - 2 * d) & (a < 1e-3), (r > 0.25 + 2 * d) & (a > 0.999)

            def pres(q, al, m):
                rho = q[0][m] / al[m]
                u, v, w = (q[x][m] / q[0][m] for x in (1, 2, 3))
                return (0.4 * (q[4][m] / al[m] - 0.5 * rho * (u * u + v * v + w * w))).mean()
            hist.append(pres(qN, 1 - a, inn) - pres(qP, a, out))
    assert o.status == 0
    return np.array(hist), I0, o


def test_static_sphere_keeps_the_laplace_jump():
    """A gas sphere started in Laplace equilibrium (p inside = p outside +
    2 sigma / R = 288 above it) keeps the jump: within 2 % over 60 steps on
    24^3 (6 cells a radius), closer than on 16^3."""
    h16, _, _ = _laplace_jump_3d(16, 60)
    h24, _, _ = _laplace_jump_3d(24, 60)
    e16, e24 = np.abs(h16 / 288.0 - 1.0).max(), np.abs(h24 / 288.0 - 1.0).max()
    assert e24 <= 0.02 and e24 < e16, (e16, e24)


def test_no_jump_without_surface_tension_and_masses_kept():
    h, _, _ = _laplace_jump_3d(16, 30, sigma=0.0, equilibrium=False)
    assert np.abs(h).max() <= 0.05 * 288.0, h
    # the accelerated cycle with surface tension keeps each fluid's mass
    _, I0, o = _laplace_jump_3d(16, 10, multi=True)
    I1 = o.integrals()
    for k in range(2):
        assert abs(I1[k, 0] - I0[k, 0]) <= 1e-13 * I0[k, 0]


# -- viscosity (Eq. 3, 5) in 3D -------------------------------------------------

def _viscous_drop_2d(n=24):
    """A gas drop in gas at one pressure with a shear flow through both
    (u = 0.5 sin(2 pi y)), both fluids viscous."""
    c = I.static_drop(n, sigma=0.0, equilibrium=False, liquid=False)
    c["cfg"]["mu"] = [0.02, 0.01]
    X, Y = I._centres(c["cfg"])
    for key in ("prim_N", "prim_P"):
        c[key][1] = 0.5 * np.sin(2.0 * math.pi * Y)
    return c


def test_viscous_step_on_z_invariant_case_is_the_2d_step():
    """Face viscous fluxes, the interface traction and their place in Eq. 2
    reduce to the 2D oracle's on a z-invariant case (fixed steps)."""
    c2 = _viscous_drop_2d()
    c3 = I.extrude(c2, 4)
    c3["cfg"]["mu"] = c2["cfg"]["mu"]
    o2 = O.Oracle(c2["cfg"]).init(c2["phi"], c2["prim_N"], c2["prim_P"])
    o3 = O.Oracle3(c3["cfg"]).init(c3["phi"], c3["prim_N"], c3["prim_P"])
    dts = [1.5e-4, 2e-4, 1.5e-4]  # below both CFL steps (viscous limit included)
    _fixed_steps(o2, dts)
    _fixed_steps(o3, dts)
    q2, q3 = o2.state(), o3.state()
    for f in range(2):
        assert np.all(q3[f][3] == 0.0)
        for z in range(4):
            for m2, m3 in ((0, 0), (1, 1), (2, 2), (3, 4)):
                # momenta against mass x the shear speed 0.5 (the y
                # momentum is small: its own scale would judge round-off
                # of the geometry's two formulas)
                ref = q2[f][m2]
                scale = max(np.abs(ref).max(), 0.5 * np.abs(q2[f][0]).max() if m2 in (1, 2) else 0.0)
                err = np.abs(q3[f][m3][z] - ref).max() / scale
                assert err < 1e-12, (f, m2, z, err)


def test_shear_wave_along_z_decays_at_the_viscous_rate():
    """u = a sin(2 pi z) in a periodic box decays as exp(-nu (2 pi)^2 t):
    the z-direction terms of the face flux (closed form)."""
    n, mu, amp = 32, 0.01, 0.01
    cfg = I.config3(4, 4, n, 1.0 / n, I.AIR, I.AIR, ["periodic"] * 6, mu=[mu, mu])
    X, Y, Z = I._centres3(cfg)
    phi = np.ones_like(X)  # fluid P everywhere
    prim = I._uniform3(X.shape, 1.0, 0.0, 0.0, 0.0, 100.0)
    prim[1] = amp * np.sin(2.0 * math.pi * Z)
    o = O.Oracle3(cfg).init(phi, prim, prim)
    T = 0.5
    o.step_single_dt(100000, t_end=T)
    qP = o.state()[1]
    u = qP[1] / qP[0]
    a = 2.0 * (u[:, 0, 0] * np.sin(2.0 * math.pi * Z[:, 0, 0])).mean()
    assert a == pytest.approx(amp * math.exp(-mu * (2.0 * math.pi) ** 2 * T), rel=2e-3)
    # nothing moves across the wave (viscous heating varies along z, so the
    # pressure it raises moves the gas along z)
    assert np.abs(qP[2]).max() == 0.0


def test_viscous_case_with_permuted_axes_gives_the_permuted_result():
    c = I.shock_bubble_3d(8)
    c["cfg"]["mu"] = [0.01, 0.005]
    cp = _permute_case(c)
    oa = O.Oracle3(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    ob = O.Oracle3(cp["cfg"]).init(cp["phi"], cp["prim_N"], cp["prim_P"])
    for o in (oa, ob):
        o.step_single_dt(2)
        o.step_multi_dt(1)
    qa, qb = oa.state(), ob.state()
    back = _permute_case({"cfg": c["cfg"], "phi": qa[2], "prim_N": qa[0], "prim_P": qa[1]})
    for f, key in ((0, "prim_N"), (1, "prim_P")):
        for m in range(5):
            assert _rel(qb[f][m], back[key][m]) < 1e-11, (f, m)
