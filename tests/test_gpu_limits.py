"""Error paths of the two bounded loops of a step, on the GPU and without
any fault: the sub-cycle limit of the accelerated cycle (Sec. 3.1's
fluid-2 loop) gives SIF_ETIMEOUT, the Newton limit of the interface
Riemann problem (Sec. 2.1's exchange flux) gives SIF_ENOCONV; both are
host-set limits on loops that end by themselves, the device records the
condition in its error word and the host reads it after the call.  The
context stays usable afterwards."""
import os

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
    return [np.ascontiguousarray(case[x]) for x in ("phi", "prim_N", "prim_P")]


def _solver(sif, case, graphs):
    """A solver whose cycles run as captured graphs (the default) or are
    issued from the host (SIF_NO_GRAPH=1 at creation)."""
    old = os.environ.get("SIF_NO_GRAPH")
    os.environ["SIF_NO_GRAPH"] = "0" if graphs else "1"
    try:
        return sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    finally:
        if old is None:
            del os.environ["SIF_NO_GRAPH"]
        else:
            os.environ["SIF_NO_GRAPH"] = old


FAST_GAS = lambda: inputs.underwater_explosion(77, radius=0.3, p_gas=1e8, rho_gas=1.0, seed=7)


@pytest.mark.parametrize("graphs", [True, False])
def test_substep_limit_gives_etimeout(graphs):
    sif = _sif()
    case = FAST_GAS()
    o = O.Oracle(case["cfg"]).init(*_arrays(case))
    need = o.step_multi_dt(1)["substeps"]
    assert need >= 3
    # a limit the cycle reaches exactly is no error
    s = _solver(sif, case, graphs)
    s.set_limits(max_substeps=need)
    assert s.step_multi_dt(1)["substeps"] == need
    # one fewer stops the cycle before its last sub-step
    s = _solver(sif, case, graphs)
    s.set_limits(max_substeps=need - 1)
    with pytest.raises(sif.SifError) as e:
        s.step_multi_dt(1)
    assert e.value.code == sif.ETIMEOUT, e.value
    # usable again after a restart with the default limit back
    s.set_limits(max_substeps=4096)
    s.init_fluids(*_arrays(case))
    assert s.step_multi_dt(1)["substeps"] == need


@pytest.mark.parametrize("graphs", [True, False])
def test_newton_limit_gives_enoconv(graphs):
    sif = _sif()
    case = inputs.shock_tube_1d(64, rk_order=2)
    s = _solver(sif, case, graphs)
    # the water/air interface's Riemann problem needs several iterations
    # from the acoustic guess (p 1e9 against 1e5 Pa): one is not enough
    s.set_limits(newton_iters=1)
    with pytest.raises(sif.SifError) as e:
        s.step_multi_dt(1)
    assert e.value.code == sif.ENOCONV, e.value
    with pytest.raises(sif.SifError) as e:
        s.step_single_dt(1)
    assert e.value.code == sif.ENOCONV
    s.set_limits(newton_iters=50)
    s.init_fluids(*_arrays(case))
    g = s.step_single_dt(1)
    o = O.Oracle(case["cfg"]).init(*_arrays(case))
    oi = o.step_single_dt(1)
    assert g["t"] == pytest.approx(oi["t"], rel=1e-14)


def test_limits_out_of_range_are_refused():
    sif = _sif()
    case = inputs.shock_tube_1d(64, rk_order=2)
    s = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    with pytest.raises(sif.SifError) as e:
        s.set_limits(max_substeps=10 ** 7)
    assert e.value.code == sif.EINVAL
    with pytest.raises(sif.SifError) as e:
        s.set_limits(newton_iters=10 ** 5)
    assert e.value.code == sif.EINVAL
