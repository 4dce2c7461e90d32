"""Parity of the CUDA path with viscosity (Eq. 3 and 5: the viscous part
of each finite-volume stage in its own kernel, each fluid's viscous
traction added to its exchange flux in the interface kernel, the explicit
viscous limit in the CFL rate) against the oracle: the shear wave in both
orientations, the 1D sound wave, the gas drop with viscosity and surface
tension, and the shock-bubble with viscosity (helium sub-cycled).  One
step or cycle to 1e-12, longer runs to 1e-8 with the same schedule; the
shear wave's decay on the GPU against exp(-nu k^2 t); the adjoint tape is
refused with viscosity."""
import math

import numpy as np
import pytest

from paper_1905_03917_gb300 import inputs
from tests.test_gpu_parity import compare, pair, sound_speed_scale

pytestmark = pytest.mark.gpu


def _drop():
    c = inputs.static_drop(64, equilibrium=True, liquid=False)
    c["cfg"] = dict(c["cfg"], mu=(0.05, 0.01))
    return c


def _shock_bubble():
    c = inputs.shock_bubble(128, 32, seed=3, perturb=1e-3)
    c["cfg"] = dict(c["cfg"], mu=(2e-4, 1e-4))
    return c


CASES = {
    "shear_y": lambda: inputs.shear_wave(32, across="y"),
    "shear_x": lambda: inputs.shear_wave(32, across="x"),
    "sound": lambda: inputs.sound_wave(64),
    "drop": _drop,
    "shock_bubble": _shock_bubble,
}
MULTI = ["drop", "shock_bubble"]


@pytest.mark.parametrize("name", list(CASES))
def test_single_steps(name):
    case = CASES[name]()
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
    case = CASES[name]()
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


def test_shear_wave_decays_at_the_viscous_rate_on_the_gpu():
    n, mu, amp, T = 32, 0.01, 0.01, 0.5
    g, _ = pair(inputs.shear_wave(n, mu=mu, amp=amp))
    g.step_single_dt(100000, T)
    assert abs(g.t - T) <= 1e-12
    _, qP, _ = g.state()
    y = (np.arange(n) + 0.5) / n
    a = 2.0 * ((qP[1] / qP[0]) * np.sin(2 * np.pi * y)[:, None]).mean()
    assert abs(a / (amp * math.exp(-mu * (2 * math.pi) ** 2 * T)) - 1.0) < 1e-3


def test_adjoint_tape_is_refused():
    from paper_1905_03917_gb300 import sif
    g, _ = pair(CASES["shear_y"]())
    with pytest.raises(sif.SifError) as e:
        g.tape_reset(4)
    assert e.value.code == sif.EINVAL
