"""The extension of Sec. 2.3 run as all its Jacobi sweeps per band tile in
shared memory (the default) against one launch per sweep or two
(SIF_EXT_SWEEPS=1): the two compute every band value by the same
operations in the same order, so whole runs agree bit for bit, on the
multi-time-step cycle and the single-step method, with the sweep count
below, at and above the tile's halo, with bands that reach the domain's
walls and its periodic seams."""
import os

import numpy as np
import pytest

from paper_1905_03917_gb300 import inputs
from tests.test_gpu_parity import _sif

pytestmark = pytest.mark.gpu


def _solver(case, per_sweep, **kw):
    sif = _sif()
    if per_sweep:
        os.environ["SIF_EXT_SWEEPS"] = "1"
    try:
        cfg = dict(case["cfg"], **kw)
        return sif.Solver(cfg).init_fluids(*(np.ascontiguousarray(case[x], dtype=np.float64)
                                             for x in ("phi", "prim_N", "prim_P")))
    finally:
        os.environ.pop("SIF_EXT_SWEEPS", None)


CASES = {
    "shock_bubble": lambda: inputs.shock_bubble(160, 40, seed=3, perturb=1e-3),
    "explosion": lambda: inputs.underwater_explosion(96, seed=5, perturb=1e-3),
    "bubble_periodic": lambda: inputs.periodic_bubble(48, seed=1),
    "tube": lambda: inputs.shock_tube_1d(203, rk_order=2, interface=0.4913),
    "droplet_tait": lambda: inputs.droplet_translation(40),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("multi", [True, False])
def test_blocked_extension_is_bitwise_the_sweeps(name, multi):
    case = CASES[name]()
    a, b = _solver(case, False), _solver(case, True)
    for _ in range(12):
        ra = a.step_multi_dt(1) if multi else a.step_single_dt(1)
        rb = b.step_multi_dt(1) if multi else b.step_single_dt(1)
        assert ra["substeps"] == rb["substeps"]
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("iters", [1, 4, 12, 13])
def test_sweep_counts(iters):
    """1 and 4 sweeps (halo narrower than the band), 12 (the widest halo
    the blocked kernel takes), 13 (beyond it: the sweeps run per launch in
    both solvers)."""
    case = inputs.shock_bubble(128, 32, seed=4, perturb=1e-3)
    a, b = _solver(case, False, ext_iters=iters), _solver(case, True, ext_iters=iters)
    for _ in range(6):
        assert a.step_multi_dt(1)["substeps"] == b.step_multi_dt(1)["substeps"]
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)
