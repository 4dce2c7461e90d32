"""The accelerated cycle with SSP-RK3 on the GPU against the oracle's
(Sec. 3.1 steps 1-5 carried to three stages; Eq. 8-9 with RK3's weights):
one cycle to 1e-12 and 100 cycles to 1e-8 with the same schedule, the
ratio-one cycle bitwise equal to the single RK3 step, conservation with
the correction, the host-issued cycle bitwise equal to the captured graph,
and a batch of RK3 instances bitwise equal to the instances alone."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs
from tests.test_gpu_parity import _sif, compare, pair

pytestmark = pytest.mark.gpu


def _rk3(case):
    case["cfg"] = dict(case["cfg"], rk_order=3)
    return case


CASES = {
    "tube": lambda: inputs.shock_tube_1d(400, rk_order=3),
    "bubble_periodic": lambda: _rk3(inputs.periodic_bubble(48, seed=1)),
    "shock_bubble": lambda: _rk3(inputs.shock_bubble(128, 32, seed=3, perturb=1e-3)),
    "explosion": lambda: _rk3(inputs.underwater_explosion(96, seed=5, perturb=1e-3)),
    "explosion_fast_gas": lambda: _rk3(inputs.underwater_explosion(77, radius=0.3, p_gas=1e8,
                                                                   rho_gas=1.0, seed=7)),
}


def _arrays(case):
    return [np.ascontiguousarray(case[x]) for x in ("phi", "prim_N", "prim_P")]


@pytest.mark.parametrize("name", list(CASES))
def test_one_rk3_cycle(name):
    g, o = pair(CASES[name]())
    gi, oi = g.step_multi_dt(1), o.step_multi_dt(1)
    assert gi["substeps"] == oi["substeps"] >= 2
    assert gi["open_updates"] == oi["open_updates"]
    compare(g, o, 1e-12)


@pytest.mark.parametrize("name", ["shock_bubble", "explosion_fast_gas", "tube"])
def test_hundred_rk3_cycles(name):
    g, o = pair(CASES[name]())
    subs_g = [g.step_multi_dt(1)["substeps"] for _ in range(100)]
    subs_o = [o.step_multi_dt(1)["substeps"] for _ in range(100)]
    assert subs_g == subs_o and max(subs_o) >= 2
    compare(g, o, 1e-8)
    assert abs(g.t - o.t) <= 1e-10 * o.t


def test_ratio_one_rk3_cycle_equals_single_step_bitwise():
    sif = _sif()
    case = CASES["bubble_periodic"]()
    a = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    b = sif.Solver(dict(case["cfg"], force_ratio_one=1)).init_fluids(*_arrays(case))
    for _ in range(10):
        a.step_single_dt(1)
        b.step_multi_dt(1)
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)


def test_rk3_cycles_conserve_on_the_gpu():
    g, _ = pair(CASES["bubble_periodic"]())
    I0 = g.integrals().sum(0)
    subs = [g.step_multi_dt(1)["substeps"] for _ in range(60)]
    assert max(subs) >= 3
    I1 = g.integrals().sum(0)
    scale = np.array([I0[0], I0[0] * 2000.0, I0[0] * 2000.0, I0[3]])
    assert (np.abs(I1 - I0) / scale).max() <= 1e-13


def test_host_issued_rk3_cycle_equals_graph():
    sif = _sif()
    case = CASES["explosion_fast_gas"]()
    a = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    old = os.environ.get("SIF_NO_GRAPH")
    os.environ["SIF_NO_GRAPH"] = "1"
    try:
        b = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    finally:
        if old is None:
            del os.environ["SIF_NO_GRAPH"]
        else:
            os.environ["SIF_NO_GRAPH"] = old
    for _ in range(5):
        assert a.step_multi_dt(1)["substeps"] == b.step_multi_dt(1)["substeps"]
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)


def test_batch_of_rk3_instances_equals_instances_alone():
    sif = _sif()
    cases = [_rk3(c) for c in inputs.batched_instances(count=6, seed=3, nmin=48, nmax=96)]
    b = sif.Batch([c["cfg"] for c in cases])
    for s, c in zip(b.instances, cases):
        s.init_fluids(*_arrays(c))
    for _ in range(3):
        assert b.step_multi_dt(1) > 0
    for s, c in zip(b.instances, cases):
        solo = sif.Solver(c["cfg"]).init_fluids(*_arrays(c))
        solo.step_multi_dt(3)
        for x, y in zip(s.state(), solo.state()):
            assert np.array_equal(x, y), c["name"]
        solo.close()
