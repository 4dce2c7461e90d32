"""Thin ctypes binding of libsif (include/sif.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  Arrays may be numpy arrays (host memory, SIF_HOST) or CUDA
torch tensors (device memory, SIF_DEVICE, passed by data_ptr()).  There
is no CPU fallback: if the library cannot be loaded this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, EINVAL, ECUDA, ENONPHYS, ENOCONV, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6
HOST, DEVICE = 0, 1
BC = {"reflect": 0, "zerograd": 1, "periodic": 2}
_NAMES = {EINVAL: "SIF_EINVAL", ECUDA: "SIF_ECUDA", ENONPHYS: "SIF_ENONPHYS",
          ENOCONV: "SIF_ENOCONV", ETIMEOUT: "SIF_ETIMEOUT", ESTATE: "SIF_ESTATE"}

EXPORTS = ["sif_create", "sif_init_fluids", "sif_step_single_dt", "sif_step_multi_dt",
           "sif_integrals", "sif_get_state", "sif_set_state", "sif_get_time",
           "sif_last_error", "sif_destroy", "sif_save", "sif_load",
           "sif_profile_enable", "sif_profile_read", "sif_measure_fp64_peak",
           "sif_integrals_noalloc", "sif_set_tile_shape", "sif_get_tile_shape",
           "sif_batch_create", "sif_batch_instance", "sif_batch_step_multi_dt",
           "sif_batch_last_error", "sif_batch_destroy", "sif_batch_one_graph",
           "sif_tape_reset", "sif_tape_length", "sif_replay_step", "sif_adjoint_step",
           "sif_adjoint_init", "sif_probe_reciprocal", "sif_set_limits",
           "sif3_create", "sif3_init_fluids", "sif3_step_single_dt", "sif3_step_multi_dt",
           "sif3_get_state", "sif3_set_state", "sif3_integrals", "sif3_geometry",
           "sif3_get_time", "sif3_profile_enable", "sif3_profile_read", "sif3_last_error",
           "sif3_destroy", "sif3_set_limits"]


class SifError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


# face fluxes of the finite-volume stage: WENO5-LF (the paper's), HLLC
FLUXES = {"lf": 0, "hllc": 1}

class Config(ctypes.Structure):
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
                ("cuda_stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("weno_char", ctypes.c_int), ("sigma", ctypes.c_double),
                ("mu", ctypes.c_double * 2), ("tait", ctypes.c_int * 2),
                ("tait_B", ctypes.c_double * 2), ("tait_rho0", ctypes.c_double * 2),
                ("tait_p0", ctypes.c_double * 2), ("flux", ctypes.c_int)]


class Config3(ctypes.Structure):
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
                ("tait_p0", ctypes.c_double * 2),
                ("cuda_stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("sigma", ctypes.c_double), ("mu", ctypes.c_double * 2)]


class Profile(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong), ("fv_launches", ctypes.c_longlong),
                ("fv_ms", ctypes.c_double), ("fv_cell_updates", ctypes.c_longlong),
                ("fv_open_updates", ctypes.c_longlong)]


class CycleInfo(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt1", ctypes.c_double), ("dt2", ctypes.c_double),
                ("n_raw", ctypes.c_double), ("n_used", ctypes.c_double),
                ("role_fluid1", ctypes.c_int), ("substeps", ctypes.c_int),
                ("cell_updates", ctypes.c_longlong), ("open_updates", ctypes.c_longlong)]


_lib = None


def load(path: str | None = None):
    """Load libsif (building it in-tree first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libsif not found at {path}")
    L = ctypes.CDLL(path)
    P, D, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    L.sif_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(P)]
    L.sif_init_fluids.argtypes = [P, P, P, P, I]
    L.sif_step_single_dt.argtypes = [P, I, D, ctypes.POINTER(CycleInfo)]
    L.sif_step_multi_dt.argtypes = [P, I, D, ctypes.POINTER(CycleInfo)]
    L.sif_integrals.argtypes = [P, P]
    L.sif_get_state.argtypes = [P, P, P, P, I]
    L.sif_set_state.argtypes = [P, P, P, P, D, I]
    L.sif_get_time.argtypes = [P, ctypes.POINTER(D)]
    L.sif_last_error.argtypes = [P]
    L.sif_last_error.restype = ctypes.c_char_p
    L.sif_destroy.argtypes = [P]
    L.sif_destroy.restype = None
    L.sif_save.argtypes = [P, P, ctypes.POINTER(ctypes.c_size_t)]
    L.sif_load.argtypes = [P, P, ctypes.c_size_t]
    L.sif_profile_enable.argtypes = [P, I]
    L.sif_profile_read.argtypes = [P, ctypes.POINTER(Profile)]
    L.sif_measure_fp64_peak.argtypes = [I, ctypes.POINTER(D)]
    L.sif_probe_reciprocal.argtypes = [P, P, ctypes.c_longlong, P]
    L.sif_integrals_noalloc.argtypes = [P, P, I, I, D, D, P, P]
    L.sif_set_tile_shape.argtypes = [P, I, I]
    L.sif_set_limits.argtypes = [P, I, I]
    L.sif_set_limits.restype = I
    L.sif_get_tile_shape.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
    L.sif_batch_create.argtypes = [I, ctypes.POINTER(Config), ctypes.POINTER(P)]
    L.sif_batch_instance.argtypes = [P, I, ctypes.POINTER(P)]
    L.sif_batch_step_multi_dt.argtypes = [P, I, ctypes.POINTER(ctypes.c_longlong),
                                          ctypes.POINTER(ctypes.c_longlong)]
    L.sif_batch_last_error.argtypes = [P]
    L.sif_batch_last_error.restype = ctypes.c_char_p
    L.sif_batch_destroy.argtypes = [P]
    L.sif_batch_destroy.restype = None
    L.sif_batch_one_graph.argtypes = [P]
    L.sif_batch_one_graph.restype = I
    L.sif_tape_reset.argtypes = [P, I]
    L.sif_tape_length.argtypes = [P, ctypes.POINTER(I)]
    L.sif_replay_step.argtypes = [P, I, P, P, I]
    L.sif_adjoint_step.argtypes = [P, I, P, P, I]
    L.sif_adjoint_init.argtypes = [P, P, P, P, P, P, I]
    L.sif3_create.argtypes = [ctypes.POINTER(Config3), ctypes.POINTER(P)]
    L.sif3_init_fluids.argtypes = [P, P, P, P, I]
    L.sif3_step_single_dt.argtypes = [P, I, D, ctypes.POINTER(CycleInfo)]
    L.sif3_step_multi_dt.argtypes = [P, I, D, ctypes.POINTER(CycleInfo)]
    L.sif3_get_state.argtypes = [P, P, P, P, I]
    L.sif3_set_state.argtypes = [P, P, P, P, I]
    L.sif3_integrals.argtypes = [P, P]
    L.sif3_geometry.argtypes = [P, P, P, P, P, P, P, P, I]
    L.sif3_get_time.argtypes = [P, ctypes.POINTER(D)]
    L.sif3_profile_enable.argtypes = [P, I]
    L.sif3_profile_read.argtypes = [P, ctypes.POINTER(Profile)]
    L.sif3_last_error.argtypes = [P]
    L.sif3_last_error.restype = ctypes.c_char_p
    L.sif3_destroy.argtypes = [P]
    L.sif3_set_limits.argtypes = [P, I, I]
    L.sif3_set_limits.restype = I
    for f in (L.sif3_create, L.sif3_init_fluids, L.sif3_step_single_dt, L.sif3_step_multi_dt,
              L.sif3_get_state, L.sif3_set_state, L.sif3_integrals, L.sif3_geometry,
              L.sif3_get_time, L.sif3_profile_enable, L.sif3_profile_read, L.sif3_destroy):
        f.restype = I
    for f in (L.sif_tape_reset, L.sif_tape_length, L.sif_replay_step, L.sif_adjoint_step,
              L.sif_adjoint_init):
        f.restype = I
    for f in (L.sif_create, L.sif_init_fluids, L.sif_step_single_dt, L.sif_step_multi_dt,
              L.sif_integrals, L.sif_get_state, L.sif_set_state, L.sif_get_time,
              L.sif_save, L.sif_load, L.sif_profile_enable, L.sif_profile_read,
              L.sif_measure_fp64_peak, L.sif_probe_reciprocal, L.sif_integrals_noalloc,
              L.sif_set_tile_shape, L.sif_get_tile_shape, L.sif_batch_create,
              L.sif_batch_instance, L.sif_batch_step_multi_dt):
        f.restype = I
    _lib = L
    return L


def make_config(cfg: dict, stream=None, device=0) -> Config:
    c = Config()
    c.dim, c.nx, c.ny = int(cfg["dim"]), int(cfg["nx"]), int(cfg["ny"])
    c.x0, c.y0 = float(cfg.get("x0", 0.0)), float(cfg.get("y0", 0.0))
    c.dx, c.dy = float(cfg["dx"]), float(cfg["dy"])
    for i, b in enumerate(cfg["bc"]):
        c.bc[i] = BC[b] if isinstance(b, str) else int(b)
    for k in range(2):
        c.gamma[k], c.pinf[k] = float(cfg["gamma"][k]), float(cfg["pinf"][k])
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
    c.cuda_stream = stream
    c.device = int(device)
    c.weno_char = int(cfg.get("weno_char", 0))
    c.sigma = float(cfg.get("sigma", 0.0))
    mu = cfg.get("mu", (0.0, 0.0))
    c.mu[0], c.mu[1] = float(mu[0]), float(mu[1])
    # face flux: "lf" (WENO5 on Lax-Friedrichs split fluxes) or "hllc"
    fl = cfg.get("flux", "lf")
    if fl not in FLUXES:
        raise ValueError(f"flux must be one of {sorted(FLUXES)}")
    c.flux = FLUXES[fl]
    # Tait's equation per fluid: (B, rho0, p0), or None for a stiffened gas
    for k, t in enumerate(cfg.get("tait", (None, None))):
        if t is not None:
            c.tait[k] = 1
            c.tait_B[k], c.tait_rho0[k], c.tait_p0[k] = (float(x) for x in t)
    return c


def _ptr(a):
    """(pointer, mem_kind) of a numpy array or a CUDA torch tensor."""
    if a is None:
        return None, HOST
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous float64")
        return a.ctypes.data, HOST
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("device tensors must be contiguous float64")
        return a.data_ptr(), DEVICE
    raise TypeError(f"unsupported array type {type(a)}")


def measure_fp64_peak(device=0) -> float:
    """Measured FP64 FMA throughput of the device in TFLOP/s."""
    v = ctypes.c_double()
    rc = load().sif_measure_fp64_peak(int(device), ctypes.byref(v))
    if rc != OK:
        raise SifError(rc, "FP64 throughput probe failed")
    return v.value


def probe_reciprocal(d):
    """The finite-volume kernel's reciprocal of every element of a
    contiguous float64 CUDA tensor (sif_probe_reciprocal), as a new tensor
    on the current stream."""
    import torch
    if not (getattr(d, "is_cuda", False) and d.dtype == torch.float64 and d.is_contiguous()):
        raise ValueError("a contiguous float64 CUDA tensor is required")
    r = torch.empty_like(d)
    stream = torch.cuda.current_stream(d.device).cuda_stream
    rc = load().sif_probe_reciprocal(d.data_ptr(), r.data_ptr(), d.numel(), stream)
    if rc != OK:
        raise SifError(rc, "reciprocal probe failed")
    return r


def integrals_noalloc(q_N, q_P, dx, dy, out, stream=None):
    """Totals of device planes (contiguous float64 CUDA tensors of shape
    (4, ny, nx)) into the device tensor `out` (at least 8 doubles) without
    any device allocation; see sif_integrals_noalloc in include/sif.h.
    All three tensors must be on one GPU; the call runs with that GPU
    current, on `stream` (a cudaStream_t handle) or, by default, on torch's
    current stream of that GPU, so that it is ordered after the work that
    filled the planes."""
    import torch
    (a, ka), (b, kb), (o, ko) = _ptr(q_N), _ptr(q_P), _ptr(out)
    if not (ka == kb == ko == DEVICE):
        raise ValueError("integrals_noalloc takes device tensors")
    if q_N.dim() != 3 or q_N.shape[0] != 4:
        raise ValueError(f"q_N must have shape (4, ny, nx), got {tuple(q_N.shape)}")
    if tuple(q_P.shape) != tuple(q_N.shape):
        raise ValueError(f"q_P has shape {tuple(q_P.shape)}, q_N {tuple(q_N.shape)}")
    if out.numel() < 8:
        raise ValueError("out must hold at least 8 doubles")
    if not (q_N.device == q_P.device == out.device):
        raise ValueError("q_N, q_P and out must be on the same GPU")
    ny, nx = q_N.shape[-2], q_N.shape[-1]
    with torch.cuda.device(q_N.device):
        st = stream if stream is not None else torch.cuda.current_stream(q_N.device).cuda_stream
        rc = load().sif_integrals_noalloc(a, b, int(nx), int(ny), float(dx), float(dy), o, st)
    if rc != OK:
        raise SifError(rc, "sif_integrals_noalloc rejected the call")


class Solver:
    """One two-fluid problem held on the GPU by libsif."""

    def __init__(self, cfg: dict, stream=None, device=0, _handle=None):
        self.cfg = dict(cfg)
        self.nx, self.ny = int(cfg["nx"]), int(cfg["ny"])
        self._owned = _handle is None
        if _handle is not None:  # an instance owned by a Batch
            self._h = _handle
            return
        L = load()
        h = ctypes.c_void_p()
        c = make_config(cfg, stream, device)
        rc = L.sif_create(ctypes.byref(c), ctypes.byref(h))
        if rc != OK:
            raise SifError(rc, "sif_create rejected the configuration or failed to allocate")
        self._h = h

    def _check(self, rc):
        if rc != OK:
            msg = load().sif_last_error(self._h).decode()
            raise SifError(rc, msg)

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                load().sif_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fluids(self, phi, prim_N, prim_P):
        (p0, k0), (p1, k1), (p2, k2) = _ptr(phi), _ptr(prim_N), _ptr(prim_P)
        if not (k0 == k1 == k2):
            raise ValueError("all inputs must be in the same memory")
        self._keep = (phi, prim_N, prim_P)
        self._check(load().sif_init_fluids(self._h, p0, p1, p2, k0))
        self._keep = None
        return self

    def _info(self, info):
        return {"t": info.t, "dt1": info.dt1, "dt2": info.dt2, "n_raw": info.n_raw,
                "n_used": info.n_used, "role_fluid1": info.role_fluid1,
                "substeps": info.substeps, "cell_updates": info.cell_updates,
                "open_updates": info.open_updates,
                "fluid_cell_updates": info.open_updates / int(self.cfg.get("rk_order", 2))}

    def step_single_dt(self, nsteps=1, t_end=0.0):
        info = CycleInfo()
        self._check(load().sif_step_single_dt(self._h, int(nsteps), float(t_end), ctypes.byref(info)))
        return self._info(info)

    def step_multi_dt(self, ncycles=1, t_end=0.0):
        info = CycleInfo()
        self._check(load().sif_step_multi_dt(self._h, int(ncycles), float(t_end), ctypes.byref(info)))
        return self._info(info)

    def integrals(self):
        out = np.empty(8)
        self._check(load().sif_integrals(self._h, out.ctypes.data))
        return out.reshape(2, 4)

    def state(self):
        n = self.nx * self.ny
        qN, qP, phi = np.empty(4 * n), np.empty(4 * n), np.empty(n)
        self._check(load().sif_get_state(self._h, qN.ctypes.data, qP.ctypes.data, phi.ctypes.data, HOST))
        sh = (4, self.ny, self.nx)
        return qN.reshape(sh), qP.reshape(sh), phi.reshape(self.ny, self.nx)

    def state_into(self, qN, qP, phi):
        (a, ka), (b, kb), (c, kc) = _ptr(qN), _ptr(qP), _ptr(phi)
        self._check(load().sif_get_state(self._h, a, b, c, ka))

    def set_state(self, qN, qP, phi, t=0.0):
        (a, ka), (b, kb), (c, kc) = _ptr(qN), _ptr(qP), _ptr(phi)
        self._check(load().sif_set_state(self._h, a, b, c, float(t), ka))

    def save(self) -> bytes:
        """Checkpoint (host bytes) of everything a bitwise continuation needs."""
        n = ctypes.c_size_t(0)
        self._check(load().sif_save(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(load().sif_save(self._h, ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(n)))
        return buf.raw[: n.value]

    def set_tile_shape(self, tx: int, ty: int):
        self._check(load().sif_set_tile_shape(self._h, int(tx), int(ty)))

    def set_limits(self, max_substeps=0, newton_iters=0):
        """Sub-steps per accelerated cycle and Newton iterations per
        interface Riemann problem (0 keeps a limit); see sif_set_limits."""
        self._check(load().sif_set_limits(self._h, int(max_substeps), int(newton_iters)))

    @property
    def tile_shape(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check(load().sif_get_tile_shape(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def profile(self, enable: bool = True):
        self._check(load().sif_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self):
        p = Profile()
        self._check(load().sif_profile_read(self._h, ctypes.byref(p)))
        return {"kernel_launches": p.kernel_launches, "fv_launches": p.fv_launches,
                "fv_ms": p.fv_ms, "fv_cell_updates": p.fv_cell_updates,
                "fv_open_updates": p.fv_open_updates}

    def load_checkpoint(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        self._check(load().sif_load(self._h, ctypes.cast(buf, ctypes.c_void_p), len(data)))
        return self

    @property
    def t(self):
        v = ctypes.c_double()
        self._check(load().sif_get_time(self._h, ctypes.byref(v)))
        return v.value

    # -- adjoint of the frozen single-dt step (sif_tape_* / sif_adjoint_*) --

    def tape_reset(self, capacity: int):
        self._check(load().sif_tape_reset(self._h, int(capacity)))

    @property
    def tape_length(self) -> int:
        v = ctypes.c_int()
        self._check(load().sif_tape_length(self._h, ctypes.byref(v)))
        return v.value

    def _pair(self, a, b):
        (pa, ka), (pb, kb) = _ptr(a), _ptr(b)
        if ka != kb:
            raise ValueError("both arrays must be in the same memory")
        n = 8 * self.nx * self.ny
        for x in (a, b):
            size = x.size if isinstance(x, np.ndarray) else x.numel()
            if size != n:
                raise ValueError(f"expected {n} doubles (2 x 4 x ny x nx)")
        return pa, pb, ka

    def replay_step(self, step, q_in, q_out=None):
        """Frozen replay of recorded step `step` from q_in (2, 4, ny, nx)."""
        if q_out is None:
            q_out = np.empty((2, 4, self.ny, self.nx))
        a, b, k = self._pair(q_in, q_out)
        self._check(load().sif_replay_step(self._h, int(step), a, b, k))
        return q_out

    def adjoint_step(self, step, lam_in, lam_out=None):
        """Adjoint of the state before recorded step `step` from that after it."""
        if lam_out is None:
            lam_out = np.empty((2, 4, self.ny, self.nx))
        a, b, k = self._pair(lam_in, lam_out)
        self._check(load().sif_adjoint_step(self._h, int(step), a, b, k))
        return lam_out

    def adjoint_init(self, phi, prim_N, prim_P, lam_q, lam_prim=None):
        """Adjoint of the primitive initial fields from that of the initial state."""
        if lam_prim is None:
            lam_prim = np.empty((2, 4, self.ny, self.nx))
        ptrs = [_ptr(x) for x in (phi, prim_N, prim_P, lam_q, lam_prim)]
        kinds = {k for _, k in ptrs}
        if len(kinds) != 1:
            raise ValueError("all arrays must be in the same memory")
        self._check(load().sif_adjoint_init(self._h, *[p for p, _ in ptrs], kinds.pop()))
        return lam_prim


class Batch:
    """Independent two-fluid problems advanced together (one graph launch
    per batch cycle; see sif_batch_* in include/sif.h)."""

    def __init__(self, cfgs, device=0):
        L = load()
        n = len(cfgs)
        arr = (Config * n)(*[make_config(c, None, device) for c in cfgs])
        h = ctypes.c_void_p()
        rc = L.sif_batch_create(n, arr, ctypes.byref(h))
        if rc != OK:
            raise SifError(rc, "sif_batch_create failed")
        self._h = h
        self.instances = []
        for i, c in enumerate(cfgs):
            ih = ctypes.c_void_p()
            rc = L.sif_batch_instance(h, i, ctypes.byref(ih))
            if rc != OK:
                raise SifError(rc, "sif_batch_instance failed")
            self.instances.append(Solver(c, _handle=ih))

    def __len__(self):
        return len(self.instances)

    def __getitem__(self, i):
        return self.instances[i]

    def step_multi_dt(self, ncycles=1):
        """ncycles batch cycles; returns the (cell, fluid) stage updates of
        all instances (active-tile cells); last_open_updates keeps the
        open-cell count of the same call."""
        n, o = ctypes.c_longlong(0), ctypes.c_longlong(0)
        rc = load().sif_batch_step_multi_dt(self._h, int(ncycles), ctypes.byref(n), ctypes.byref(o))
        if rc != OK:
            raise SifError(rc, load().sif_batch_last_error(self._h).decode())
        self.last_open_updates = o.value
        return n.value

    @property
    def one_graph(self) -> bool:
        return bool(load().sif_batch_one_graph(self._h))

    def close(self):
        if getattr(self, "_h", None):
            for s in self.instances:
                s._h = None
            load().sif_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_config3(cfg: dict, stream=None, device=0) -> Config3:
    c = Config3()
    c.nx, c.ny, c.nz = int(cfg["nx"]), int(cfg["ny"]), int(cfg["nz"])
    c.x0, c.y0, c.z0 = (float(cfg.get(k, 0.0)) for k in ("x0", "y0", "z0"))
    c.dx, c.dy, c.dz = float(cfg["dx"]), float(cfg["dy"]), float(cfg["dz"])
    if len(cfg["bc"]) != 6:
        raise ValueError("a 3D configuration lists six boundary kinds")
    for i, b in enumerate(cfg["bc"]):
        c.bc[i] = BC[b] if isinstance(b, str) else int(b)
    for k in range(2):
        c.gamma[k], c.pinf[k] = float(cfg["gamma"][k]), float(cfg["pinf"][k])
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
    c.cuda_stream = stream
    c.device = int(device)
    c.sigma = float(cfg.get("sigma", 0.0))
    mu = cfg.get("mu", (0.0, 0.0))
    c.mu[0], c.mu[1] = float(mu[0]), float(mu[1])
    return c


class Solver3:
    """One two-fluid problem in three dimensions held on the GPU by libsif
    (include/sif3d.h).  Arrays are (nz, ny, nx), x fastest; the primitive
    fields are (rho, u, v, w, p) and the state (alpha U) has five
    components (mass, x-, y-, z-momentum, energy) per fluid."""

    def __init__(self, cfg: dict, stream=None, device=0):
        self.cfg = dict(cfg)
        self.shape = (int(cfg["nz"]), int(cfg["ny"]), int(cfg["nx"]))
        L = load()
        h = ctypes.c_void_p()
        c = make_config3(cfg, stream, device)
        rc = L.sif3_create(ctypes.byref(c), ctypes.byref(h))
        if rc != OK:
            raise SifError(rc, "sif3_create rejected the configuration or failed to allocate")
        self._h = h

    def _check(self, rc):
        if rc != OK:
            raise SifError(rc, load().sif3_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().sif3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fluids(self, phi, prim_N, prim_P):
        (p0, k0), (p1, k1), (p2, k2) = _ptr(phi), _ptr(prim_N), _ptr(prim_P)
        if not (k0 == k1 == k2):
            raise ValueError("all inputs must be in the same memory")
        n = int(np.prod(self.shape))
        for a, m in ((phi, 1), (prim_N, 5), (prim_P, 5)):
            size = a.size if isinstance(a, np.ndarray) else a.numel()
            if size != m * n:
                raise ValueError(f"expected {m} planes of {self.shape}")
        self._check(load().sif3_init_fluids(self._h, p0, p1, p2, k0))
        return self

    def _info(self, info):
        return {"t": info.t, "dt1": info.dt1, "dt2": info.dt2, "n_raw": info.n_raw,
                "n_used": info.n_used, "role_fluid1": info.role_fluid1,
                "substeps": info.substeps, "cell_updates": info.cell_updates,
                "open_updates": info.open_updates,
                "fluid_cell_updates": info.open_updates / 2}

    def step_single_dt(self, nsteps=1, t_end=0.0):
        info = CycleInfo()
        self._check(load().sif3_step_single_dt(self._h, int(nsteps), float(t_end),
                                               ctypes.byref(info)))
        return self._info(info)

    def step_multi_dt(self, ncycles=1, t_end=0.0):
        info = CycleInfo()
        self._check(load().sif3_step_multi_dt(self._h, int(ncycles), float(t_end),
                                              ctypes.byref(info)))
        return self._info(info)

    def state(self):
        n = int(np.prod(self.shape))
        qN, qP, phi = np.empty(5 * n), np.empty(5 * n), np.empty(n)
        self._check(load().sif3_get_state(self._h, qN.ctypes.data, qP.ctypes.data,
                                          phi.ctypes.data, HOST))
        sh = (5,) + self.shape
        return qN.reshape(sh), qP.reshape(sh), phi.reshape(self.shape)

    def state_into(self, qN, qP, phi):
        (a, ka), (b, kb), (c, kc) = _ptr(qN), _ptr(qP), _ptr(phi)
        self._check(load().sif3_get_state(self._h, a, b, c, ka))

    def set_state(self, qN, qP, phi):
        (a, ka), (b, kb), (c, kc) = _ptr(qN), _ptr(qP), _ptr(phi)
        self._check(load().sif3_set_state(self._h, a, b, c, ka))

    def integrals(self):
        out = np.empty(10)
        self._check(load().sif3_integrals(self._h, out.ctypes.data))
        return out.reshape(2, 5)

    def geometry(self):
        n = int(np.prod(self.shape))
        arrs = [np.empty(n) for _ in range(7)]
        self._check(load().sif3_geometry(self._h, *(a.ctypes.data for a in arrs), HOST))
        names = ("alpha", "ax", "ay", "az", "sx", "sy", "sz")
        return {k: a.reshape(self.shape) for k, a in zip(names, arrs)}

    @property
    def t(self):
        v = ctypes.c_double()
        self._check(load().sif3_get_time(self._h, ctypes.byref(v)))
        return v.value

    def set_limits(self, max_substeps=0, newton_iters=0):
        """Limits of the sub-cycle loop and the interface Newton iteration
        (<= 0 keeps a limit); see sif3_set_limits."""
        self._check(load().sif3_set_limits(self._h, int(max_substeps), int(newton_iters)))

    def profile_enable(self, on=True):
        self._check(load().sif3_profile_enable(self._h, int(bool(on))))

    def profile_read(self):
        p = Profile()
        self._check(load().sif3_profile_read(self._h, ctypes.byref(p)))
        return {"kernel_launches": p.kernel_launches, "fv_launches": p.fv_launches,
                "fv_ms": p.fv_ms, "fv_cell_updates": p.fv_cell_updates,
                "fv_open_updates": p.fv_open_updates}
