"""ctypes front end of the serial FP64 CPU oracle (``oracle/sif_oracle.c``
and its three-dimensional form ``oracle/sif_oracle3d.c``).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  Nothing here is
shared with the CUDA library or its Python binding.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sif_oracle.c")
_SRC3 = os.path.join(_HERE, "sif_oracle3d.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")

BC = {"reflect": 0, "zerograd": 1, "periodic": 2}
ERR_NONPHYS, ERR_NOCONV, ERR_INVAL = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile the oracle as a shared library (gcc, no FMA contraction)."""
    deps = [_SRC, _SRC3] + [os.path.join(_HERE, h) for h in ("sif_oracle.h", "sif_oracle3d.h")]
    newest = max(os.path.getmtime(d) for d in deps)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, _SRC, _SRC3, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


# face fluxes of the finite-volume stage: WENO5-LF (the paper's), HLLC
FLUXES = {"lf": 0, "hllc": 1}

class _Config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("bc", ctypes.c_int * 4),
                ("gamma", ctypes.c_double * 2), ("pinf", ctypes.c_double * 2),
                ("cfl", ctypes.c_double), ("rk_order", ctypes.c_int),
                ("weno_eps", ctypes.c_double), ("mix_alpha", ctypes.c_double),
                ("ratio_threshold", ctypes.c_double),
                ("ext_iters", ctypes.c_int), ("reinit_iters", ctypes.c_int),
                ("band", ctypes.c_double),
                ("flux_correction", ctypes.c_int), ("force_ratio_one", ctypes.c_int),
                ("weno_char", ctypes.c_int), ("sigma", ctypes.c_double),
                ("mu", ctypes.c_double * 2), ("tait", ctypes.c_int * 2),
                ("tait_B", ctypes.c_double * 2), ("tait_rho0", ctypes.c_double * 2),
                ("tait_p0", ctypes.c_double * 2), ("flux", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt1", ctypes.c_double), ("dt2", ctypes.c_double),
                ("n_raw", ctypes.c_double), ("n_used", ctypes.c_double),
                ("role_fluid1", ctypes.c_int), ("substeps", ctypes.c_int),
                ("err", ctypes.c_int), ("open_updates", ctypes.c_longlong)]


class _Config3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("bc", ctypes.c_int * 6),
                ("gamma", ctypes.c_double * 2), ("pinf", ctypes.c_double * 2),
                ("cfl", ctypes.c_double), ("weno_eps", ctypes.c_double),
                ("mix_alpha", ctypes.c_double), ("ratio_threshold", ctypes.c_double),
                ("ext_iters", ctypes.c_int), ("reinit_iters", ctypes.c_int),
                ("band", ctypes.c_double),
                ("flux_correction", ctypes.c_int), ("force_ratio_one", ctypes.c_int),
                ("tait", ctypes.c_int * 2),
                ("tait_B", ctypes.c_double * 2), ("tait_rho0", ctypes.c_double * 2),
                ("tait_p0", ctypes.c_double * 2), ("sigma", ctypes.c_double),
                ("mu", ctypes.c_double * 2)]


_lib_handle = None


def lib():
    global _lib_handle
    if _lib_handle is None:
        L = ctypes.CDLL(build())
        P, D, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_create.restype = P
        L.orc_create.argtypes = [ctypes.POINTER(_Config)]
        L.orc_destroy.argtypes = [P]
        L.orc_init.argtypes = [P, dp, dp, dp]
        L.orc_step_single_dt.argtypes = [P, I, D, ctypes.POINTER(_Info)]
        L.orc_step_multi_dt.argtypes = [P, I, D, ctypes.POINTER(_Info)]
        L.orc_get_state.argtypes = [P, dp, dp, dp]
        L.orc_set_state.argtypes = [P, dp, dp, dp]
        L.orc_integrals.argtypes = [P, dp]
        L.orc_time.restype = D
        L.orc_time.argtypes = [P]
        L.orc_status.argtypes = [P]
        L.orc_geometry.argtypes = [P, dp, dp, dp, dp, dp]
        L.orc_rhs.argtypes = [P, I, dp]
        L.orc_stencil_states.argtypes = [P, I, dp]
        L.orc_reinit_only.argtypes = [P]
        L.orc_mix_only.argtypes = [P, I]
        L.orc_weno5.restype = D
        L.orc_weno5.argtypes = [dp, D]
        L.orc_edge_fraction.restype = D
        L.orc_edge_fraction.argtypes = [D, D]
        L.orc_cell_alpha.restype = D
        L.orc_cell_alpha.argtypes = [D, D, D, D]
        L.orc_riemann.argtypes = [dp, dp, dp]
        L.orc_char_basis.argtypes = [D, D, D, D, D, D, I, dp, dp]
        L.orc_hllc.argtypes = [dp, dp, D, D, I, dp]
        L.orc_riemann_jump.argtypes = [dp, dp, D, dp]
        L.orc_riemann_jump2.argtypes = [dp, dp, D, I, I, dp]
        L.orc_curvature.restype = D
        L.orc_curvature.argtypes = [P, I, I]
        L.orc_step_taped.argtypes = [P, dp, dp, dp, dp]
        L.orc_replay_step.argtypes = [P, D, dp, dp, dp]
        L.orc_adjoint_step.argtypes = [P, D, dp, dp, dp, dp, dp]
        L.orc_rhs_frozen.argtypes = [P, dp, dp]
        L.orc_rhs_adjoint.argtypes = [P, dp, dp, dp]
        L.orc_mix_adjoint.argtypes = [P, I, dp]
        L.orc_adjoint_init.argtypes = [P, dp, dp, dp, dp]
        L.orc_weno5_grad.restype = None
        L.orc_weno5_grad.argtypes = [dp, D, dp]
        L.orc_riemann_grad.argtypes = [dp, dp, D, D, dp, dp]
        L.orc3_create.restype = P
        L.orc3_create.argtypes = [ctypes.POINTER(_Config3)]
        L.orc3_destroy.argtypes = [P]
        L.orc3_init.argtypes = [P, dp, dp, dp]
        L.orc3_step_single_dt.argtypes = [P, I, D, ctypes.POINTER(_Info)]
        L.orc3_step_multi_dt.argtypes = [P, I, D, ctypes.POINTER(_Info)]
        L.orc3_get_state.argtypes = [P, dp, dp, dp]
        L.orc3_set_state.argtypes = [P, dp, dp, dp]
        L.orc3_integrals.argtypes = [P, dp]
        L.orc3_geometry.argtypes = [P, dp, dp, dp, dp, dp, dp, dp]
        L.orc3_cell_alpha.restype = D
        L.orc3_cell_alpha.argtypes = [dp, dp]
        L.orc3_curvature.restype = D
        L.orc3_curvature.argtypes = [P, I, I, I]
        L.orc3_time.restype = D
        L.orc3_time.argtypes = [P]
        L.orc3_status.argtypes = [P]
        _lib_handle = L
    return _lib_handle


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_config(cfg: dict) -> _Config:
    c = _Config()
    c.dim = int(cfg["dim"])
    c.nx, c.ny = int(cfg["nx"]), int(cfg["ny"])
    c.x0, c.y0 = float(cfg.get("x0", 0.0)), float(cfg.get("y0", 0.0))
    c.dx, c.dy = float(cfg["dx"]), float(cfg["dy"])
    for i, b in enumerate(cfg["bc"]):
        c.bc[i] = BC[b] if isinstance(b, str) else int(b)
    for k in range(2):
        c.gamma[k] = float(cfg["gamma"][k])
        c.pinf[k] = float(cfg["pinf"][k])
    c.cfl = float(cfg.get("cfl", 0.6))
    c.rk_order = int(cfg.get("rk_order", 2))
    c.weno_eps = float(cfg.get("weno_eps", 1e-6))
    c.mix_alpha = float(cfg.get("mix_alpha", 0.5))
    c.ratio_threshold = float(cfg.get("ratio_threshold", 0.7))
    c.ext_iters = int(cfg.get("ext_iters", 10))
    c.reinit_iters = int(cfg.get("reinit_iters", 2))
    c.band = float(cfg.get("band", 6.0))
    c.flux_correction = int(cfg.get("flux_correction", 1))
    c.force_ratio_one = int(cfg.get("force_ratio_one", 0))
    c.weno_char = int(cfg.get("weno_char", 0))
    c.sigma = float(cfg.get("sigma", 0.0))
    mu = cfg.get("mu", (0.0, 0.0))
    c.mu[0], c.mu[1] = float(mu[0]), float(mu[1])
    # face flux: "lf" (WENO5 on Lax-Friedrichs split fluxes) or "hllc"
    fl = cfg.get("flux", "lf")
    if fl not in FLUXES:
        raise ValueError(f"flux must be one of {sorted(FLUXES)}")
    c.flux = FLUXES[fl]
    # Tait's equation per fluid: (B, rho0, p0) or None for a stiffened gas
    for k, t in enumerate(cfg.get("tait", (None, None))):
        if t is not None:
            c.tait[k] = 1
            c.tait_B[k], c.tait_rho0[k], c.tait_p0[k] = (float(x) for x in t)
    return c


class Oracle:
    """One two-fluid problem advanced by the serial oracle."""

    def __init__(self, cfg: dict):
        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        self._h = lib().orc_create(ctypes.byref(self._c))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self.nx, self.ny = self._c.nx, self._c.ny

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def init(self, phi, prim_N, prim_P):
        phi, pN, pP = _f64(phi), _f64(prim_N), _f64(prim_P)
        lib().orc_init(self._h, _ptr(phi), _ptr(pN), _ptr(pP))
        return self

    def _info(self, info):
        return {"t": info.t, "dt1": info.dt1, "dt2": info.dt2, "n_raw": info.n_raw,
                "n_used": info.n_used, "role_fluid1": info.role_fluid1,
                "substeps": info.substeps, "err": info.err,
                "open_updates": info.open_updates,
                "fluid_cell_updates": info.open_updates / self._c.rk_order}

    def step_single_dt(self, nsteps=1, t_end=0.0):
        info = _Info()
        lib().orc_step_single_dt(self._h, int(nsteps), float(t_end), ctypes.byref(info))
        return self._info(info)

    def step_multi_dt(self, ncycles=1, t_end=0.0):
        info = _Info()
        lib().orc_step_multi_dt(self._h, int(ncycles), float(t_end), ctypes.byref(info))
        return self._info(info)

    def state(self):
        n = self.nx * self.ny
        qN, qP, phi = np.empty(4 * n), np.empty(4 * n), np.empty(n)
        lib().orc_get_state(self._h, _ptr(qN), _ptr(qP), _ptr(phi))
        sh = (4, self.ny, self.nx)
        return qN.reshape(sh), qP.reshape(sh), phi.reshape(self.ny, self.nx)

    def set_state(self, qN, qP, phi):
        qN, qP, phi = _f64(qN), _f64(qP), _f64(phi)
        lib().orc_set_state(self._h, _ptr(qN), _ptr(qP), _ptr(phi))

    def integrals(self):
        out = np.empty(8)
        lib().orc_integrals(self._h, _ptr(out))
        return out.reshape(2, 4)

    @property
    def t(self):
        return lib().orc_time(self._h)

    @property
    def status(self):
        return lib().orc_status(self._h)

    def curvature(self, i, j):
        return lib().orc_curvature(self._h, int(i), int(j))

    def geometry(self):
        nx, ny = self.nx, self.ny
        al, sx, sy = np.empty(nx * ny), np.empty(nx * ny), np.empty(nx * ny)
        ax, ay = np.empty((nx + 1) * ny), np.empty(nx * (ny + 1))
        lib().orc_geometry(self._h, _ptr(al), _ptr(ax), _ptr(ay), _ptr(sx), _ptr(sy))
        return {"alpha": al.reshape(ny, nx), "ax": ax.reshape(ny, nx + 1),
                "ay": ay.reshape(ny + 1, nx), "sx": sx.reshape(ny, nx),
                "sy": sy.reshape(ny, nx)}

    def rhs(self, k):
        out = np.empty(4 * self.nx * self.ny)
        lib().orc_rhs(self._h, int(k), _ptr(out))
        return out.reshape(4, self.ny, self.nx)

    def stencil_states(self, k):
        out = np.empty(4 * self.nx * self.ny)
        lib().orc_stencil_states(self._h, int(k), _ptr(out))
        return out.reshape(4, self.ny, self.nx)

    def reinit_only(self):
        lib().orc_reinit_only(self._h)

    def mix_only(self, k):
        lib().orc_mix_only(self._h, int(k))

    # -- frozen-schedule step and its adjoint (RK2 single-dt) --

    def step_taped(self):
        """One single-dt step; returns its schedule {dt, lf[8], phi1, phi2}."""
        n = self.nx * self.ny
        dt = np.zeros(1)
        lf, phi1, phi2 = np.empty(8), np.empty(n), np.empty(n)
        rc = lib().orc_step_taped(self._h, _ptr(dt), _ptr(lf), _ptr(phi1), _ptr(phi2))
        if rc:
            raise RuntimeError(f"oracle step failed: {rc}")
        sh = (self.ny, self.nx)
        return {"dt": float(dt[0]), "lf": lf, "phi1": phi1.reshape(sh), "phi2": phi2.reshape(sh)}

    def replay_step(self, rec):
        lf, p1, p2 = _f64(rec["lf"]), _f64(rec["phi1"]), _f64(rec["phi2"])
        return lib().orc_replay_step(self._h, float(rec["dt"]), _ptr(lf), _ptr(p1), _ptr(p2))

    def rhs_frozen(self, lf):
        """L of both fluids (2, 4, ny, nx) with LF speeds lf[4] given."""
        lf, out = _f64(lf), np.empty(8 * self.nx * self.ny)
        lib().orc_rhs_frozen(self._h, _ptr(lf), _ptr(out))
        return out.reshape(2, 4, self.ny, self.nx)

    def rhs_adjoint(self, lf, mu):
        lf, mu = _f64(lf), _f64(mu)
        out = np.empty_like(mu)
        lib().orc_rhs_adjoint(self._h, _ptr(lf), _ptr(mu), _ptr(out))
        return out.reshape(2, 4, self.ny, self.nx)

    def mix_adjoint(self, k, lam):
        lam = _f64(lam).copy()
        lib().orc_mix_adjoint(self._h, int(k), _ptr(lam))
        return lam.reshape(4, self.ny, self.nx)

    def adjoint_init(self, prim_N, prim_P, lam):
        """Adjoint of the state after init -> adjoint of the primitive fields
        (2, 4, ny, nx), at the current level set."""
        pN, pP, li = _f64(prim_N), _f64(prim_P), _f64(lam)
        out = np.empty(8 * self.nx * self.ny)
        lib().orc_adjoint_init(self._h, _ptr(pN), _ptr(pP), _ptr(li), _ptr(out))
        return out.reshape(2, 4, self.ny, self.nx)

    def adjoint_step(self, rec, lam):
        """lam (2, 4, ny, nx) adjoint of the state after the step -> adjoint of
        the state before it (the current state)."""
        lf, p1, p2 = _f64(rec["lf"]), _f64(rec["phi1"]), _f64(rec["phi2"])
        li = _f64(lam)
        lo = np.empty_like(li)
        rc = lib().orc_adjoint_step(self._h, float(rec["dt"]), _ptr(lf), _ptr(p1), _ptr(p2),
                                    _ptr(li), _ptr(lo))
        if rc:
            raise RuntimeError(f"oracle adjoint failed: {rc}")
        return lo.reshape(2, 4, self.ny, self.nx)


def make_config3(cfg: dict) -> _Config3:
    c = _Config3()
    c.nx, c.ny, c.nz = int(cfg["nx"]), int(cfg["ny"]), int(cfg["nz"])
    c.x0, c.y0, c.z0 = (float(cfg.get(k, 0.0)) for k in ("x0", "y0", "z0"))
    c.dx, c.dy, c.dz = float(cfg["dx"]), float(cfg["dy"]), float(cfg["dz"])
    for i, b in enumerate(cfg["bc"]):
        c.bc[i] = BC[b] if isinstance(b, str) else int(b)
    for k in range(2):
        c.gamma[k] = float(cfg["gamma"][k])
        c.pinf[k] = float(cfg["pinf"][k])
    c.cfl = float(cfg.get("cfl", 0.6))
    c.weno_eps = float(cfg.get("weno_eps", 1e-6))
    c.mix_alpha = float(cfg.get("mix_alpha", 0.5))
    c.ratio_threshold = float(cfg.get("ratio_threshold", 0.7))
    c.ext_iters = int(cfg.get("ext_iters", 10))
    c.reinit_iters = int(cfg.get("reinit_iters", 2))
    c.band = float(cfg.get("band", 6.0))
    c.flux_correction = int(cfg.get("flux_correction", 1))
    c.force_ratio_one = int(cfg.get("force_ratio_one", 0))
    for k, t in enumerate(cfg.get("tait", (None, None))):
        if t is not None:
            c.tait[k] = 1
            c.tait_B[k], c.tait_rho0[k], c.tait_p0[k] = (float(x) for x in t)
    c.sigma = float(cfg.get("sigma", 0.0))
    mu = cfg.get("mu", (0.0, 0.0))
    c.mu[0], c.mu[1] = float(mu[0]), float(mu[1])
    return c


class Oracle3:
    """One two-fluid problem in three dimensions advanced by the serial
    oracle; arrays are (nz, ny, nx), x fastest, and the primitive fields
    (rho, u, v, w, p)."""

    def __init__(self, cfg: dict):
        self.cfg = dict(cfg)
        self._c = make_config3(cfg)
        self._h = lib().orc3_create(ctypes.byref(self._c))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self.shape = (self._c.nz, self._c.ny, self._c.nx)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc3_destroy(h)
            self._h = None

    def init(self, phi, prim_N, prim_P):
        phi, pN, pP = _f64(phi), _f64(prim_N), _f64(prim_P)
        lib().orc3_init(self._h, _ptr(phi), _ptr(pN), _ptr(pP))
        return self

    def _info(self, info):
        return {"t": info.t, "dt1": info.dt1, "dt2": info.dt2, "n_raw": info.n_raw,
                "n_used": info.n_used, "role_fluid1": info.role_fluid1,
                "substeps": info.substeps, "err": info.err,
                "open_updates": info.open_updates,
                "fluid_cell_updates": info.open_updates / 2}

    def step_single_dt(self, nsteps=1, t_end=0.0):
        info = _Info()
        lib().orc3_step_single_dt(self._h, int(nsteps), float(t_end), ctypes.byref(info))
        return self._info(info)

    def step_multi_dt(self, ncycles=1, t_end=0.0):
        info = _Info()
        lib().orc3_step_multi_dt(self._h, int(ncycles), float(t_end), ctypes.byref(info))
        return self._info(info)

    def state(self):
        n = int(np.prod(self.shape))
        qN, qP, phi = np.empty(5 * n), np.empty(5 * n), np.empty(n)
        lib().orc3_get_state(self._h, _ptr(qN), _ptr(qP), _ptr(phi))
        return qN.reshape((5,) + self.shape), qP.reshape((5,) + self.shape), phi.reshape(self.shape)

    def set_state(self, qN, qP, phi):
        qN, qP, phi = _f64(qN), _f64(qP), _f64(phi)
        lib().orc3_set_state(self._h, _ptr(qN), _ptr(qP), _ptr(phi))

    def integrals(self):
        out = np.empty(10)
        lib().orc3_integrals(self._h, _ptr(out))
        return out.reshape(2, 5)

    def geometry(self):
        n = int(np.prod(self.shape))
        arrs = [np.empty(n) for _ in range(7)]
        lib().orc3_geometry(self._h, *(_ptr(a) for a in arrs))
        names = ("alpha", "ax", "ay", "az", "sx", "sy", "sz")
        return {k: a.reshape(self.shape) for k, a in zip(names, arrs)}

    def curvature(self, i, j, k):
        return lib().orc3_curvature(self._h, int(i), int(j), int(k))

    @property
    def t(self):
        return lib().orc3_time(self._h)

    @property
    def status(self):
        return lib().orc3_status(self._h)


def cell_alpha3(corners):
    """Volume fraction and unit-face interface vector of the unit cube from
    its corner values c[i + 2 j + 4 k]."""
    c, s = _f64(corners), np.empty(3)
    a = lib().orc3_cell_alpha(_ptr(c), _ptr(s))
    return a, s


def weno5(v, eps=1e-6):
    a = _f64(v)
    return lib().orc_weno5(_ptr(a), float(eps))


def weno5_grad(v, eps=1e-6):
    a, g = _f64(v), np.empty(5)
    lib().orc_weno5_grad(_ptr(a), float(eps), _ptr(g))
    return g


def riemann_grad(left, right, lam_p, lam_u):
    """Row vector lam_p dp* + lam_u du* over (rho, u, p) of each side."""
    L, R, gL, gR = _f64(left), _f64(right), np.empty(3), np.empty(3)
    lib().orc_riemann_grad(_ptr(L), _ptr(R), float(lam_p), float(lam_u), _ptr(gL), _ptr(gR))
    return gL, gR


def edge_fraction(a, b):
    return lib().orc_edge_fraction(float(a), float(b))


def cell_alpha(c00, c10, c11, c01):
    return lib().orc_cell_alpha(float(c00), float(c10), float(c11), float(c01))


def char_basis(gamma, pinf, rho, u, v, p, d):
    """(L, R): left and right eigenvectors of the Euler flux Jacobian in
    direction d (0 = x, 1 = y), R's columns the fields (un - c, un, un,
    un + c), both 4 x 4 over the conserved components (rho, rho u, rho v, E)."""
    L, R = np.empty(16), np.empty(16)
    rc = lib().orc_char_basis(float(gamma), float(pinf), float(rho), float(u), float(v),
                              float(p), int(d), _ptr(L), _ptr(R))
    if rc:
        raise ValueError("non-physical state")
    return L.reshape(4, 4), R.reshape(4, 4)


def riemann_jump(left, right, jump):
    """As riemann() with the left star pressure exceeding the right one by
    jump; p is the right star pressure, p_L the left one."""
    L, R, out = _f64(left), _f64(right), np.empty(8)
    rc = lib().orc_riemann_jump(_ptr(L), _ptr(R), float(jump), _ptr(out))
    return {"p": out[0], "u": out[1], "rho_L": out[2], "rho_R": out[3],
            "c_L": out[4], "c_R": out[5], "iters": int(out[6]), "p_L": out[7], "rc": rc}


def hllc(WL, WR, gamma, pinf, d):
    """HLLC flux of direction d between primitive states (rho, u, v, p);
    None for a non-physical state."""
    L, R, F = _f64(WL), _f64(WR), np.empty(4)
    rc = lib().orc_hllc(_ptr(L), _ptr(R), float(gamma), float(pinf), int(d), _ptr(F))
    return None if rc else F


def riemann(left, right):
    """left/right = (rho, u, p, gamma, pinf); returns dict of the star state."""
    L, R, out = _f64(left), _f64(right), np.empty(7)
    rc = lib().orc_riemann(_ptr(L), _ptr(R), _ptr(out))
    return {"p": out[0], "u": out[1], "rho_L": out[2], "rho_R": out[3],
            "c_L": out[4], "c_R": out[5], "iters": int(out[6]), "rc": rc}


def riemann_baro(left, right, baro_l, baro_r, jump=0.0):
    """As riemann_jump() with either side barotropic (Tait's equation: the
    shock branch from mass and momentum alone, the star density on the
    fluid's curve p + pinf ~ rho^gamma)."""
    L, R, out = _f64(left), _f64(right), np.empty(8)
    rc = lib().orc_riemann_jump2(_ptr(L), _ptr(R), float(jump), int(baro_l), int(baro_r),
                                 _ptr(out))
    return {"p": out[0], "u": out[1], "rho_L": out[2], "rho_R": out[3],
            "c_L": out[4], "c_R": out[5], "iters": int(out[6]), "p_L": out[7], "rc": rc}
