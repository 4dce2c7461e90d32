"""Parity of the CUDA path's characteristic-wise WENO5 option
(`weno_char = 1`: the Lax-Friedrichs split fluxes of each face's stencil
are projected on the left eigenvectors of the face state, reconstructed
field by field and mapped back) with the oracle's: one step or cycle to
1e-12, fifty steps or thirty cycles to the long-run bar 1e-8 with the same
sub-step schedule, on the 1D tube, the shock-bubble, the explosion and the
periodic bubble; results independent of the tile shape, bitwise; the
adjoint refused in this mode."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs
from tests.test_gpu_parity import compare, pair, sound_speed_scale

pytestmark = pytest.mark.gpu

CASES = {
    "tube_rk3": lambda: inputs.shock_tube_1d(400, rk_order=3),
    "tube_rk2": lambda: inputs.shock_tube_1d(203, rk_order=2, interface=0.4913),
    "shock_bubble": lambda: inputs.shock_bubble(128, 32, seed=3, perturb=1e-3),
    "explosion": lambda: inputs.underwater_explosion(96, seed=5, perturb=1e-3),
    "explosion_fast_gas": lambda: inputs.underwater_explosion(77, radius=0.3, p_gas=1e8,
                                                              rho_gas=1.0, seed=7),
    "bubble_periodic": lambda: inputs.periodic_bubble(48, seed=1),
}
MULTI = ["tube_rk2", "shock_bubble", "explosion", "explosion_fast_gas", "bubble_periodic"]


def _char(case):
    case = dict(case)
    case["cfg"] = dict(case["cfg"], weno_char=1)
    return case


@pytest.mark.parametrize("name", list(CASES))
def test_single_steps(name):
    case = _char(CASES[name]())
    cref = sound_speed_scale(case)
    g, o = pair(case)
    g.step_single_dt(1)
    o.step_single_dt(1)
    compare(g, o, 1e-12, cref=cref)
    g.step_single_dt(49)
    o.step_single_dt(49)
    assert o.status == 0
    assert abs(g.t - o.t) <= 1e-10 * o.t
    print(name, "relative L1 after 50 steps:", compare(g, o, 1e-8, cref=cref))


@pytest.mark.parametrize("name", MULTI)
def test_multi_dt_cycles(name):
    case = _char(CASES[name]())
    cref = sound_speed_scale(case)
    g, o = pair(case)
    a, b = g.step_multi_dt(1), o.step_multi_dt(1)
    assert a["substeps"] == b["substeps"]
    compare(g, o, 1e-12, cref=cref)
    for _ in range(29):
        a, b = g.step_multi_dt(1), o.step_multi_dt(1)
        assert a["substeps"] == b["substeps"]
    assert o.status == 0
    print(name, "relative L1 after 30 cycles:", compare(g, o, 1e-8, cref=cref))


@pytest.mark.parametrize("shape", [(32, 4), (16, 8), (16, 16), (64, 4)])
def test_results_do_not_depend_on_tile_shape(shape):
    from paper_1905_03917_gb300 import sif
    case = _char(CASES["explosion_fast_gas"]())
    g0, _ = pair(case)
    g1, _ = pair(case)
    g1.set_tile_shape(*shape)
    g0.step_multi_dt(3)
    g1.step_multi_dt(3)
    for x, y in zip(g0.state(), g1.state()):
        assert np.array_equal(x, y)


def test_adjoint_tape_is_refused():
    from paper_1905_03917_gb300 import sif
    case = _char(CASES["explosion"]())
    g, _ = pair(case)
    with pytest.raises(sif.SifError) as e:
        g.tape_reset(4)
    assert e.value.code == sif.EINVAL
