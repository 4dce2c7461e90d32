"""Seeded synthetic two-fluid initial conditions.

Shared by the CUDA path's tests/bench and by the oracle's tests: it holds
no arithmetic of the method itself, only initial data (level set, and the
primitive fields rho, u, v, p of each fluid over the whole grid).  Fluid N
occupies phi < 0, fluid P occupies phi >= 0.

Every case is a dict ``{"name", "cfg", "phi", "prim_N", "prim_P"}`` with
``phi`` of shape (ny, nx) and ``prim_*`` of shape (4, ny, nx), x fastest.
The workloads are the paper's class of problems (Sec. 4.1-4.2: gas-water
shock tubes and bubbles) with stiffened-gas materials.
"""
from __future__ import annotations

import math

import numpy as np

WATER = {"gamma": 4.4, "pinf": 6.0e8}
AIR = {"gamma": 1.4, "pinf": 0.0}
HELIUM = {"gamma": 1.67, "pinf": 0.0}


def config(nx, ny, dx, dy, matN, matP, bc, dim=2, x0=0.0, y0=0.0, **kw):
    cfg = {"dim": dim, "nx": nx, "ny": ny, "x0": x0, "y0": y0, "dx": dx, "dy": dy,
           "bc": list(bc), "gamma": [matN["gamma"], matP["gamma"]],
           "pinf": [matN["pinf"], matP["pinf"]], "cfl": 0.6, "rk_order": 2,
           "weno_eps": 1e-6, "mix_alpha": 0.5, "ratio_threshold": 0.7,
           "ext_iters": 10, "reinit_iters": 2, "band": 6.0,
           "flux_correction": 1, "force_ratio_one": 0}
    if "tait" in matN or "tait" in matP:
        cfg["tait"] = [matN.get("tait"), matP.get("tait")]
    cfg.update(kw)
    return cfg


def tait(B, rho0, p0, gamma):
    """A fluid closed by Tait's equation (Eq. 4), p = B ((rho/rho0)^gamma -
    1) + p0; its sound speed is the stiffened gas's with p_inf = B - p0."""
    return {"gamma": gamma, "pinf": B - p0, "tait": (B, rho0, p0)}


def _centres(cfg):
    x = cfg["x0"] + (np.arange(cfg["nx"]) + 0.5) * cfg["dx"]
    y = cfg["y0"] + (np.arange(cfg["ny"]) + 0.5) * cfg["dy"]
    return np.meshgrid(x, y)  # (ny, nx) each


def _uniform(shape, rho, u, v, p):
    out = np.empty((4,) + shape)
    out[0], out[1], out[2], out[3] = rho, u, v, p
    return out


def _smooth_noise(rng, X, Y, amp, modes=3):
    """Sum of a few random-phase sine modes, relative amplitude amp."""
    if amp == 0.0:
        return np.zeros_like(X)
    Lx = X.max() - X.min() + 1e-300
    Ly = Y.max() - Y.min() + 1e-300
    f = np.zeros_like(X)
    for _ in range(modes):
        kx, ky = rng.integers(1, 4, size=2)
        ph = rng.uniform(0, 2 * np.pi, size=2)
        f += np.sin(2 * np.pi * kx * X / Lx + ph[0]) * np.cos(2 * np.pi * ky * Y / Ly + ph[1])
    return amp * f / modes


def normal_shock(gamma, rho1, p1, mach):
    """Post-shock state behind a normal shock of Mach `mach` running into
    gas at rest (rho1, p1): returns (rho2, u2, p2, shock speed)."""
    g, M2 = gamma, mach * mach
    c1 = math.sqrt(g * p1 / rho1)
    p2 = p1 * (1.0 + 2.0 * g / (g + 1.0) * (M2 - 1.0))
    rho2 = rho1 * (g + 1.0) * M2 / ((g - 1.0) * M2 + 2.0)
    s = mach * c1
    u2 = s * (1.0 - rho1 / rho2)
    return rho2, u2, p2, s


def shock_tube_1d(n=400, rk_order=3, interface=0.5):
    """Water (left, p = 1e9 Pa) against air (right, p = 1e5 Pa) on [0, 1] m."""
    dx = 1.0 / n
    cfg = config(n, 1, dx, dx, WATER, AIR, ["zerograd"] * 4, dim=1, rk_order=rk_order)
    x = (np.arange(n) + 0.5) * dx
    phi = (x - interface)[None, :]
    pN = _uniform((1, n), 1000.0, 0.0, 0.0, 1.0e9)
    pP = _uniform((1, n), 1.0, 0.0, 0.0, 1.0e5)
    return {"name": f"shock_tube_1d_{n}", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


def shock_bubble(nx=1024, ny=256, seed=None, perturb=0.0):
    """Air-helium shock-bubble interaction, nondimensional: [0,4]x[0,1],
    helium bubble R = 0.2 at (1, 0.5), Mach 1.22 shock at x = 0.7 moving +x.
    Zero-gradient left/right, reflective top/bottom."""
    dx, dy = 4.0 / nx, 1.0 / ny
    cfg = config(nx, ny, dx, dy, HELIUM, AIR,
                 ["zerograd", "zerograd", "reflect", "reflect"])
    X, Y = _centres(cfg)
    rng = np.random.default_rng(seed)
    cx, cy, R = 1.0, 0.5, 0.2
    if seed is not None:
        cx += rng.uniform(-2, 2) * dx
        cy += rng.uniform(-2, 2) * dy
        R += rng.uniform(-2, 2) * min(dx, dy)
    phi = np.sqrt((X - cx) ** 2 + (Y - cy) ** 2) - R
    pN = _uniform(X.shape, 0.138, 0.0, 0.0, 1.0)
    rho2, u2, p2, _ = normal_shock(1.4, 1.0, 1.0, 1.22)
    post = X < 0.7
    pP = _uniform(X.shape, 1.0, 0.0, 0.0, 1.0)
    pP[0][post], pP[1][post], pP[3][post] = rho2, u2, p2
    if perturb:
        for arr in (pN, pP):
            arr[0] *= 1.0 + _smooth_noise(rng, X, Y, perturb)
            arr[3] *= 1.0 + _smooth_noise(rng, X, Y, perturb)
    return {"name": f"shock_bubble_{nx}x{ny}", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


def underwater_explosion(n=2048, seed=None, perturb=0.0, half=1.0, radius=0.12,
                         centre=(0.0, 0.0), p_gas=8.29e8, rho_gas=1270.0):
    """Gas bubble (gamma 1.4, rho 1270, p 8.29e8 Pa) of radius 0.12 m in
    water (p 1e5 Pa) on [-1,1]^2 m, reflective walls."""
    d = 2.0 * half / n
    cfg = config(n, n, d, d, AIR, WATER, ["reflect"] * 4, x0=-half, y0=-half)
    X, Y = _centres(cfg)
    rng = np.random.default_rng(seed)
    cx, cy, R = centre[0], centre[1], radius
    if seed is not None:
        cx += rng.uniform(-2, 2) * d
        cy += rng.uniform(-2, 2) * d
        R += rng.uniform(-2, 2) * d
    phi = np.sqrt((X - cx) ** 2 + (Y - cy) ** 2) - R
    pN = _uniform(X.shape, rho_gas, 0.0, 0.0, p_gas)
    pP = _uniform(X.shape, 1000.0, 0.0, 0.0, 1.0e5)
    if perturb:
        for arr in (pN, pP):
            arr[0] *= 1.0 + _smooth_noise(rng, X, Y, perturb)
            arr[3] *= 1.0 + _smooth_noise(rng, X, Y, perturb)
    return {"name": f"underwater_explosion_{n}", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


# reference scales of the nondimensional gas-water units: rho_ref = 1000
# kg/m^3, p_ref = 1e9 Pa, L_ref = 1 m (so u_ref = 1000 m/s, t_ref = 1 ms)
RHO_REF, P_REF = 1000.0, 1.0e9
WATER_ND = {"gamma": 4.4, "pinf": 6.0e8 / P_REF}


def adjoint_bubble(n=512, centre=(0.0, 0.0), radius=0.12, p_gas=8.29e8, rho_gas=1270.0,
                   seed=None):
    """Gas bubble in water on [-1,1]^2 with reflective walls (the
    underwater-explosion setup at reduced size) in nondimensional units
    (rho / 1000 kg/m^3, p / 1e9 Pa, lengths in m), in which the states and
    fluxes are of order one.  The gradient of the wall-pressure functional
    is taken with respect to this case's initial gas pressure."""
    d = 2.0 / n
    cfg = config(n, n, d, d, AIR, WATER_ND, ["reflect"] * 4, x0=-1.0, y0=-1.0)
    X, Y = _centres(cfg)
    rng = np.random.default_rng(seed)
    cx, cy, R = centre[0], centre[1], radius
    if seed is not None:
        cx += rng.uniform(-1, 1) * d
        cy += rng.uniform(-1, 1) * d
    phi = np.sqrt((X - cx) ** 2 + (Y - cy) ** 2) - R
    pN = _uniform(X.shape, rho_gas / RHO_REF, 0.0, 0.0, p_gas / P_REF)
    pP = _uniform(X.shape, 1.0, 0.0, 0.0, 1.0e5 / P_REF)
    return {"name": f"adjoint_bubble_{n}", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


def periodic_bubble(n=64, seed=0, ratio=100.0, perturb=1e-2, velocity=5.0):
    """All-periodic unit box, gas bubble in water with smooth random
    perturbations of density, pressure and velocity (conservation tests)."""
    d = 1.0 / n
    cfg = config(n, n, d, d, AIR, WATER, ["periodic"] * 4)
    X, Y = _centres(cfg)
    rng = np.random.default_rng(seed)
    cx, cy = 0.5 + rng.uniform(-2, 2) * d, 0.5 + rng.uniform(-2, 2) * d
    R = 0.2 + rng.uniform(-2, 2) * d
    phi = np.sqrt((X - cx) ** 2 + (Y - cy) ** 2) - R
    pN = _uniform(X.shape, 1.0, 0.0, 0.0, ratio * 1e5)
    pP = _uniform(X.shape, 1000.0, 0.0, 0.0, 1e5)
    for arr in (pN, pP):
        arr[0] *= 1.0 + _smooth_noise(rng, X, Y, perturb)
        arr[3] *= 1.0 + _smooth_noise(rng, X, Y, perturb)
        arr[1] = velocity * _smooth_noise(rng, X, Y, 1.0)
        arr[2] = velocity * _smooth_noise(rng, X, Y, 1.0)
    return {"name": f"periodic_bubble_{n}", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


def static_interface(nx=32, ny=32, angle=0.0, offset=0.013, p=1.0e5):
    """Planar interface between water-like and gas-like stiffened gases at
    rest with uniform pressure; reflective box of unit size."""
    dx, dy = 1.0 / nx, 1.0 / ny
    matN = {"gamma": 1.4, "pinf": 0.0}
    matP = {"gamma": 4.4, "pinf": 6.0e8}
    cfg = config(nx, ny, dx, dy, matN, matP, ["reflect"] * 4)
    X, Y = _centres(cfg)
    nvec = (math.cos(angle), math.sin(angle))
    phi = (X - 0.5) * nvec[0] + (Y - 0.5) * nvec[1] - offset
    pN = _uniform(X.shape, 1.2, 0.0, 0.0, p)
    pP = _uniform(X.shape, 1000.0, 0.0, 0.0, p)
    return {"name": "static_interface", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


def single_fluid(nx=32, ny=32, seed=0, amp=0.1):
    """Whole domain filled by fluid P (phi > 0 everywhere): periodic smooth
    flow for the single-fluid reduction of the cut-cell update."""
    dx, dy = 1.0 / nx, 1.0 / ny
    cfg = config(nx, ny, dx, dy, AIR, AIR, ["periodic"] * 4)
    X, Y = _centres(cfg)
    rng = np.random.default_rng(seed)
    phi = np.ones_like(X)
    pP = _uniform(X.shape, 1.0, 0.5, -0.25, 1.0)
    pP[0] *= 1.0 + _smooth_noise(rng, X, Y, amp)
    pP[3] *= 1.0 + _smooth_noise(rng, X, Y, amp)
    pN = pP.copy()
    return {"name": "single_fluid", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


def batched_instances(count=256, seed=0, nmin=64, nmax=512):
    """Independent gas-water bubble instances of uneven sizes: N uniform in
    [nmin, nmax], bubble radius U[0.05, 0.3] (at least four cells from the
    walls), bubble/water pressure ratio log-uniform in [10, 1e4], gas
    density 1, on [-1,1]^2 with reflective walls."""
    out = []
    for s in range(count):
        rng = np.random.default_rng([seed, s])
        n = int(rng.integers(nmin, nmax + 1))
        R = float(rng.uniform(0.05, 0.3))
        ratio = float(10.0 ** rng.uniform(1.0, 4.0))
        d = 2.0 / n
        lim = 1.0 - R - 4.0 * d
        cx, cy = (float(v) for v in rng.uniform(-lim, lim, size=2))
        case = underwater_explosion(n=n, radius=R, centre=(cx, cy),
                                    p_gas=ratio * 1.0e5, rho_gas=1.0)
        case["name"] = f"instance_{s}_{n}"
        out.append(case)
    return out


def degenerate(kind, seed=0):
    """Geometries at the edges of the cut-cell rules, gas (fluid N) against
    water (fluid P, at ten times the pressure; the water's sound speed about
    five times the gas's, so the water steps are sub-cycled) at rest in a
    reflective box:

    * ``face``: a vertical interface exactly on a column of cell faces, so
      the corner values on it are exactly zero (ties count as fluid P);
    * ``diagonal``: a 45-degree interface through cell centres and corners
      (phi exactly zero at both) on a square grid;
    * ``saddle``: gas in two opposite quadrants around a point inside a
      cell (phi the signed distance to the two lines), so that the corner
      values of the cells around that point alternate in sign (four edge
      crossings);
    * ``tiny``: a 5 x 3 grid, smaller than one finite-volume tile, holding
      a gas pocket of radius 0.3 (1.5 cells in x, 0.9 in y);
    * ``film``: a gas layer 0.8 to 1.8 cells thick across the box, so that
      most interface cells are small cells of one fluid or the other.
    """
    n = {"face": (32, 12), "diagonal": (24, 24), "saddle": (26, 22), "tiny": (5, 3),
         "film": (40, 30)}[kind]
    nx, ny = n
    dx, dy = 1.0 / nx, 1.0 / ny
    matN = {"gamma": 1.4, "pinf": 0.0}
    cfg = config(nx, ny, dx, dy, matN, WATER, ["reflect"] * 4)
    X, Y = _centres(cfg)
    rng = np.random.default_rng(seed)
    if kind == "face":
        phi = X - 0.5
    elif kind == "diagonal":
        # (i - j) dx from integers: exact zeros, and exactly antisymmetric
        # under the reflection (x, y) -> (1 - y, 1 - x)
        phi = (np.arange(nx)[None, :] - np.arange(ny)[:, None]) * dx
    elif kind == "saddle":
        xc, yc = 0.5 + 0.3 * dx, 0.5 + 0.2 * dy
        phi = np.where((X - xc) * (Y - yc) > 0, -1.0, 1.0) * np.minimum(abs(X - xc), abs(Y - yc))
    elif kind == "tiny":
        phi = np.hypot(X - 0.45, Y - 0.5) - 0.3
    else:
        thick = (1.3 + 0.5 * np.sin(2 * np.pi * X + rng.uniform(0, 2 * np.pi))) * dy
        phi = np.abs(Y - 0.5) - 0.5 * thick
    pN = _uniform(X.shape, 1.2, 0.0, 0.0, 1.0e5)
    pP = _uniform(X.shape, 1000.0, 0.0, 0.0, 1.0e6)
    return {"name": f"degenerate_{kind}", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


def static_drop(n=64, sigma=36.0, equilibrium=False, liquid=True):
    """The static drop of Sec. 4.3 (Laplace law): a drop of radius 0.1
    (fluid N, phi = r - 0.1) at the centre of the unit box in air, both at
    rest at p0 = 1e3, surface tension sigma = 36, so that the pressure jump
    tends to sigma / R = 360.  The paper's Tait liquid (rho0 = 1000, B =
    5e5, gamma = 7.15) is the isentrope of a stiffened gas with gamma 7.15
    and p_inf = B - p0; air is an ideal gas (gamma 1.4, rho 1).  liquid=False
    makes the drop a gas too (gamma 1.4, rho 10): its rho c^2 is ~1000 times
    smaller, so the pressure noise of sub-cell interface motion stays far
    below the Laplace jump.  Reflective walls stand in for the paper's
    no-slip walls (no viscosity here).  equilibrium=True starts the drop at
    p0 + sigma / R instead of p0."""
    d = 1.0 / n
    p0 = 1.0e3
    matN = {"gamma": 7.15, "pinf": 5.0e5 - p0} if liquid else {"gamma": 1.4, "pinf": 0.0}
    matP = {"gamma": 1.4, "pinf": 0.0}
    cfg = config(n, n, d, d, matN, matP, ["reflect"] * 4, sigma=sigma)
    X, Y = _centres(cfg)
    phi = np.hypot(X - 0.5, Y - 0.5) - 0.1
    pN = _uniform(X.shape, 1000.0 if liquid else 10.0, 0.0, 0.0,
                  p0 + (sigma / 0.1 if equilibrium else 0.0))
    pP = _uniform(X.shape, 1.0, 0.0, 0.0, p0)
    return {"name": f"static_drop_{'liquid' if liquid else 'gas'}_{n}", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


def shear_wave(n=32, m=8, mu=0.01, amp=0.01, p=100.0, across="y"):
    """Decaying shear wave in one viscous gas (fluid P everywhere) at
    uniform density 1 and pressure p on a periodic box of n cells across
    the wave (length 1) and m along it: u = amp sin(2 pi y), v = 0
    (across="y") or v = amp sin(2 pi x), u = 0 (across="x").  The velocity
    varies across the wave only, so u_t = nu u_yy (or v_t = nu v_xx) holds
    exactly and the amplitude decays as exp(-nu (2 pi)^2 t), nu = mu."""
    d = 1.0 / n
    nx, ny = (m, n) if across == "y" else (n, m)
    cfg = config(nx, ny, d, d, AIR, AIR, ["periodic"] * 4, mu=(mu, mu))
    X, Y = _centres(cfg)
    phi = np.ones_like(X)
    pP = _uniform(X.shape, 1.0, 0.0, 0.0, p)
    if across == "y":
        pP[1] = amp * np.sin(2 * np.pi * Y)
    else:
        pP[2] = amp * np.sin(2 * np.pi * X)
    return {"name": f"shear_wave_{across}_{n}", "cfg": cfg, "phi": phi, "prim_N": pP.copy(),
            "prim_P": pP}


def sound_wave(n=32, mu=0.01, amp=1e-3, p=100.0):
    """Standing sound wave u = amp c sin(2 pi x) in one viscous gas (1D,
    periodic, density 1, pressure p): with Stokes' hypothesis and no heat
    conduction its amplitude decays as exp(-(2/3) nu k^2 t), k = 2 pi."""
    d = 1.0 / n
    cfg = config(n, 1, d, d, AIR, AIR, ["periodic"] * 4, dim=1, mu=(mu, mu))
    X, _ = _centres(cfg)
    phi = np.ones_like(X)
    c = math.sqrt(1.4 * p)
    pP = _uniform(X.shape, 1.0, 0.0, 0.0, p)
    pP[1] = amp * c * np.sin(2 * np.pi * X)
    return {"name": f"sound_wave_{n}", "cfg": cfg, "phi": phi, "prim_N": pP.copy(), "prim_P": pP}


def _square_sdf(X, Y, cx, cy, half):
    """Euclidean signed distance to the square |x - cx|, |y - cy| <= half
    (negative inside)."""
    dx, dy = np.abs(X - cx) - half, np.abs(Y - cy) - half
    outside = np.hypot(np.maximum(dx, 0.0), np.maximum(dy, 0.0))
    inside = np.minimum(np.maximum(dx, dy), 0.0)
    return outside + inside


def _ellipse_sdf(X, Y, cx, cy, a, b, samples=200000):
    """Signed distance to the ellipse ((x - cx)/a)^2 + ((y - cy)/b)^2 = 1
    (negative inside), from the nearest of densely sampled boundary points
    refined by Newton's method on the parametric angle."""
    from scipy.spatial import cKDTree
    t = np.linspace(0.0, 2.0 * np.pi, samples, endpoint=False)
    tree = cKDTree(np.stack([a * np.cos(t), b * np.sin(t)], axis=1))
    px, py = (X - cx).ravel(), (Y - cy).ravel()
    _, idx = tree.query(np.stack([px, py], axis=1))
    th = t[idx]
    for _ in range(8):  # stationary point of the squared distance in theta
        ex, ey = a * np.cos(th), b * np.sin(th)
        dx_, dy_ = -a * np.sin(th), b * np.cos(th)
        g = (ex - px) * dx_ + (ey - py) * dy_
        h = dx_ * dx_ + dy_ * dy_ + (ex - px) * (-a * np.cos(th)) + (ey - py) * (-b * np.sin(th))
        th = th - g / np.where(np.abs(h) > 1e-30, h, 1e-30)
    d = np.hypot(a * np.cos(th) - px, b * np.sin(th) - py)
    inside = (px / a) ** 2 + (py / b) ** 2 < 1.0
    return np.where(inside, -d, d).reshape(X.shape)


def circle_recovery(n=64):
    """Sec. 4.4: a 0.2 x 0.2 square drop of a Tait liquid (rho0 = 1000, B =
    5e5, gamma = 7.15, p0 = 1e3, mu = 1e-3; fluid N) in a Tait gas-like
    fluid (rho0 = 1, B = 100, gamma = 1.4, p0 = 1e3, mu = 1.6e-5) on the
    unit box, surface tension 73, both at rest at their reference states.
    The drop relaxes to a circle of the same area, R = sqrt(0.04/pi), whose
    Laplace jump is sigma/R = 646.94566.  phi is the Euclidean signed
    distance to the square (the paper reinitialises its max-norm form
    first); reflective walls stand in for the no-slip ones (the drop never
    reaches them)."""
    d = 1.0 / n
    liq, gas = tait(5.0e5, 1000.0, 1.0e3, 7.15), tait(100.0, 1.0, 1.0e3, 1.4)
    cfg = config(n, n, d, d, liq, gas, ["reflect"] * 4, sigma=73.0, mu=(1.0e-3, 1.6e-5))
    X, Y = _centres(cfg)
    phi = _square_sdf(X, Y, 0.5, 0.5, 0.1)
    pN = _uniform(X.shape, 1000.0, 0.0, 0.0, 1.0e3)
    pP = _uniform(X.shape, 1.0, 0.0, 0.0, 1.0e3)
    return {"name": f"circle_recovery_{n}", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


def drop_oscillation(n=64, a=0.2, b=0.125):
    """Sec. 4.5: an elliptic drop of a Tait liquid (rho0 = 100, B = 2e5,
    gamma = 7.15, p0 = 1e4; fluid N) at rest in a Tait gas-like fluid
    (rho0 = 1, B = 500, gamma = 1.4, p0 = 1e4), surface tension 341.642, no
    viscosity, on the unit box.  Semi-axes a = 0.2 and b = 0.125 give the
    equilibrium radius R = sqrt(a b) = 0.158 that the paper's period
    T = 0.0878 of the Rayleigh mode o = 2 belongs to (its printed minor
    axis, 0.12, would give R = 0.155).  phi is the signed distance to the
    ellipse."""
    d = 1.0 / n
    liq, gas = tait(2.0e5, 100.0, 1.0e4, 7.15), tait(500.0, 1.0, 1.0e4, 1.4)
    cfg = config(n, n, d, d, liq, gas, ["reflect"] * 4, sigma=341.642)
    X, Y = _centres(cfg)
    phi = _ellipse_sdf(X, Y, 0.5, 0.5, a, b)
    pN = _uniform(X.shape, 100.0, 0.0, 0.0, 1.0e4)
    pP = _uniform(X.shape, 1.0, 0.0, 0.0, 1.0e4)
    return {"name": f"drop_oscillation_{n}", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


def droplet_translation(n=64):
    """Sec. 4.2 (the paper's Table 1 case): a water droplet of radius 0.1
    (Tait's equation, B = 3310, rho0 = 1000, p0 = 1, gamma = 7.15; fluid N)
    at the centre of the periodic unit box in air (ideal gas, rho 1.2,
    gamma 1.4), both at p = 1 moving with u = sqrt(10)/100, v = 0
    (nondimensional: p / 1 atm, rho / 1 kg/m^3).  One period of the
    translation takes t = 10 sqrt(10)."""
    d = 1.0 / n
    water = tait(3310.0, 1000.0, 1.0, 7.15)
    cfg = config(n, n, d, d, water, AIR, ["periodic"] * 4)
    X, Y = _centres(cfg)
    phi = np.hypot(X - 0.5, Y - 0.5) - 0.1
    u = math.sqrt(10.0) / 100.0
    pN = _uniform(X.shape, 1000.0, u, 0.0, 1.0)
    pP = _uniform(X.shape, 1.2, u, 0.0, 1.0)
    return {"name": f"droplet_translation_{n}", "cfg": cfg, "phi": phi, "prim_N": pN,
            "prim_P": pP}


def gas_water_tube(n=200):
    """Sec. 4.1's gas-water shock tube: high-pressure gas (rho 0.01, p 1000,
    gamma 2, ideal) for x < 0.5 against Tait water (rho 1, p 1, gamma 7.15,
    B = 3310, rho0 = 1, p0 = 1), nondimensional, zero-gradient ends; the
    paper runs it to t = 0.0008."""
    d = 1.0 / n
    gas = {"gamma": 2.0, "pinf": 0.0}
    water = tait(3310.0, 1.0, 1.0, 7.15)
    cfg = config(n, 1, d, d, gas, water, ["zerograd"] * 4, dim=1)
    x = (np.arange(n) + 0.5) * d
    phi = (x - 0.5)[None, :]
    pN = _uniform((1, n), 0.01, 0.0, 0.0, 1000.0)
    pP = _uniform((1, n), 1.0, 0.0, 0.0, 1.0)
    return {"name": f"gas_water_tube_{n}", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


# -- three-dimensional cases (Tables 1, 3, 4, "Uniform grid - 3D") -----------
# Arrays are (nz, ny, nx), x fastest; prim_* holds (rho, u, v, w, p).

def config3(nx, ny, nz, d, matN, matP, bc, **kw):
    """Configuration of a 3D case on cubic cells of edge d; bc lists the six
    sides -x, +x, -y, +y, -z, +z."""
    cfg = {"dim": 3, "nx": nx, "ny": ny, "nz": nz, "x0": 0.0, "y0": 0.0, "z0": 0.0,
           "dx": d, "dy": d, "dz": d, "bc": list(bc),
           "gamma": [matN["gamma"], matP["gamma"]], "pinf": [matN["pinf"], matP["pinf"]],
           "cfl": 0.6, "weno_eps": 1e-6, "mix_alpha": 0.5, "ratio_threshold": 0.7,
           "ext_iters": 10, "reinit_iters": 2, "band": 6.0, "flux_correction": 1,
           "force_ratio_one": 0}
    if "tait" in matN or "tait" in matP:
        cfg["tait"] = [matN.get("tait"), matP.get("tait")]
    cfg.update(kw)
    return cfg


def _centres3(cfg):
    x = cfg["x0"] + (np.arange(cfg["nx"]) + 0.5) * cfg["dx"]
    y = cfg["y0"] + (np.arange(cfg["ny"]) + 0.5) * cfg["dy"]
    z = cfg["z0"] + (np.arange(cfg["nz"]) + 0.5) * cfg["dz"]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def _uniform3(shape, rho, u, v, w, p):
    out = np.empty((5,) + shape)
    out[0], out[1], out[2], out[3], out[4] = rho, u, v, w, p
    return out


def droplet_translation_3d(n=128):
    """Sec. 4.2's 3D case (Table 1, 128^3): the water droplet of
    droplet_translation() as a sphere, phi = |x - (0.5, 0.5, 0.5)| - 0.1, in
    the periodic unit cube, both fluids moving with u = sqrt(10)/100, v = w =
    0 at p = 1."""
    d = 1.0 / n
    water = tait(3310.0, 1000.0, 1.0, 7.15)
    cfg = config3(n, n, n, d, water, AIR, ["periodic"] * 6)
    X, Y, Z = _centres3(cfg)
    phi = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) - 0.1
    u = math.sqrt(10.0) / 100.0
    pN = _uniform3(X.shape, 1000.0, u, 0.0, 0.0, 1.0)
    pP = _uniform3(X.shape, 1.2, u, 0.0, 0.0, 1.0)
    return {"name": f"droplet_translation_3d_{n}", "cfg": cfg, "phi": phi, "prim_N": pN,
            "prim_P": pP}


def shock_bubble_3d(n=32, seed=None, perturb=0.0):
    """A 3D air-helium shock-bubble on a 2n x n x n box of edge 1/n: a
    helium sphere of radius 0.25 at (0.75, 0.5, 0.5) (fluid N) hit by a Mach
    1.22 shock in air moving in +x from x = 0.3; zero-gradient x ends,
    reflective y and z walls; seeded smooth perturbation of the sphere's
    radius."""
    d = 1.0 / n
    cfg = config3(2 * n, n, n, d, HELIUM, AIR,
                  ["zerograd", "zerograd", "reflect", "reflect", "reflect", "reflect"])
    X, Y, Z = _centres3(cfg)
    r = 0.25
    if seed is not None and perturb:
        rng = np.random.default_rng(seed)
        th = np.arctan2(Z - 0.5, Y - 0.5)
        r = r * (1.0 + perturb * np.cos(rng.integers(2, 5) * th + rng.uniform(0, 2 * np.pi)))
    phi = np.sqrt((X - 0.75) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) - r
    rho2, u2, p2, _ = normal_shock(1.4, 1.0, 1.0, 1.22)
    pre = X >= 0.3
    pP = _uniform3(X.shape, 1.0, 0.0, 0.0, 0.0, 1.0)
    pP[0][~pre], pP[1][~pre], pP[4][~pre] = rho2, u2, p2
    pN = _uniform3(X.shape, 0.138, 0.0, 0.0, 0.0, 1.0)
    return {"name": f"shock_bubble_3d_{2 * n}x{n}x{n}", "cfg": cfg, "phi": phi,
            "prim_N": pN, "prim_P": pP}


def extrude(case, nz):
    """A 2D case repeated along z over nz cells of the x spacing, periodic
    in z, with w = 0: the 3D method must reproduce the 2D one on it."""
    c2 = case["cfg"]
    bc = list(c2["bc"])
    kw = {k: c2[k] for k in ("cfl", "weno_eps", "mix_alpha", "ratio_threshold", "ext_iters",
                             "reinit_iters", "band", "flux_correction", "force_ratio_one")
          if k in c2}
    mats = [{"gamma": c2["gamma"][k], "pinf": c2["pinf"][k]} for k in range(2)]
    if "tait" in c2:
        for k in range(2):
            if c2["tait"][k] is not None:
                mats[k]["tait"] = tuple(c2["tait"][k])
    cfg = config3(c2["nx"], c2["ny"], nz, c2["dx"], mats[0], mats[1],
                  bc + ["periodic", "periodic"], **kw)
    cfg["dy"] = c2["dy"]

    def rep(a):
        return np.repeat(a[..., None, :, :], nz, axis=-3)

    def prim(p2):
        out = np.zeros((5, nz) + p2.shape[1:])
        out[0], out[1], out[2], out[4] = rep(p2[0]), rep(p2[1]), rep(p2[2]), rep(p2[3])
        return out

    return {"name": case["name"] + f"_z{nz}", "cfg": cfg, "phi": rep(case["phi"]),
            "prim_N": prim(case["prim_N"]), "prim_P": prim(case["prim_P"])}


def static_drop_3d(n=24, sigma=36.0, radius=0.25, equilibrium=True):
    """Sec. 4.3's static drop as a sphere: a gas drop (gamma 1.4, rho 10;
    fluid N) of radius 0.25 at the centre of the unit cube in air (gamma
    1.4, rho 1), both at rest at p0 = 1e3, surface tension sigma, so that
    the pressure jump tends to 2 sigma / R (Laplace's law for a sphere);
    equilibrium=True starts the drop at p0 + 2 sigma / R.  Reflective
    walls."""
    d = 1.0 / n
    p0 = 1.0e3
    gas = {"gamma": 1.4, "pinf": 0.0}
    cfg = config3(n, n, n, d, gas, AIR, ["reflect"] * 6, sigma=sigma)
    X, Y, Z = _centres3(cfg)
    phi = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) - radius
    pN = _uniform3(X.shape, 10.0, 0.0, 0.0, 0.0,
                   p0 + (2.0 * sigma / radius if equilibrium else 0.0))
    pP = _uniform3(X.shape, 1.0, 0.0, 0.0, 0.0, p0)
    return {"name": f"static_drop_3d_{n}", "cfg": cfg, "phi": phi, "prim_N": pN, "prim_P": pP}


def circle_recovery_3d(n=128):
    """Sec. 4.4's 3D case (Table 3, 128^3): circle_recovery()'s Tait liquid
    as a cube of half-width 0.1 at the centre of the unit cube in the Tait
    gas-like fluid, surface tension 73, both viscous, at rest; the drop
    relaxes to a sphere.  phi is the Euclidean signed distance to the cube
    (the paper reinitialises its max-norm form first); reflective walls."""
    d = 1.0 / n
    liq, gas = tait(5.0e5, 1000.0, 1.0e3, 7.15), tait(100.0, 1.0, 1.0e3, 1.4)
    cfg = config3(n, n, n, d, liq, gas, ["reflect"] * 6, sigma=73.0, mu=(1.0e-3, 1.6e-5))
    X, Y, Z = _centres3(cfg)
    q = [np.abs(A - 0.5) - 0.1 for A in (X, Y, Z)]
    outside = np.sqrt(sum(np.maximum(qa, 0.0) ** 2 for qa in q))
    inside = np.minimum(np.maximum(np.maximum(q[0], q[1]), q[2]), 0.0)
    phi = outside + inside
    pN = _uniform3(X.shape, 1000.0, 0.0, 0.0, 0.0, 1.0e3)
    pP = _uniform3(X.shape, 1.0, 0.0, 0.0, 0.0, 1.0e3)
    return {"name": f"circle_recovery_3d_{n}", "cfg": cfg, "phi": phi, "prim_N": pN,
            "prim_P": pP}


def filament_3d(n=64):
    """Sec. 4.6's 3D case (Table 4, 64 x 64 x 128): a liquid filament of
    radius R = 0.19 mm with a hemispherical cap, its half-length to the
    cap's centre 1.52 mm, in one eighth of the physical domain (1 x 1 x 2
    mm; reflective symmetry planes at x = y = z = 0 and walls opposite), SI
    units.  Tait liquid (rho0 = 1000, p0 = 1e4, B = 3e6, gamma = 7.15, mu =
    1e-3; fluid N) in Tait air (rho0 = 1, p0 = 1e4, B = 500, gamma = 1.4, mu
    = 1.6e-5), surface tension 0.072, both at rest."""
    mm = 1.0e-3
    d = mm / n
    liq, gas = tait(3.0e6, 1000.0, 1.0e4, 7.15), tait(500.0, 1.0, 1.0e4, 1.4)
    cfg = config3(n, n, 2 * n, d, liq, gas, ["reflect"] * 6, sigma=0.072,
                  mu=(1.0e-3, 1.6e-5))
    X, Y, Z = _centres3(cfg)
    zc = 1.52 * mm
    phi = np.where(Z < zc, np.sqrt(X ** 2 + Y ** 2),
                   np.sqrt(X ** 2 + Y ** 2 + (Z - zc) ** 2)) - 0.19 * mm
    pN = _uniform3(X.shape, 1000.0, 0.0, 0.0, 0.0, 1.0e4)
    pP = _uniform3(X.shape, 1.0, 0.0, 0.0, 0.0, 1.0e4)
    return {"name": f"filament_3d_{n}x{n}x{2 * n}", "cfg": cfg, "phi": phi, "prim_N": pN,
            "prim_P": pP}
