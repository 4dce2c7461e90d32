"""Longer GPU-against-oracle runs over seeded geometries: gas bubbles of
random size, position (down to four cells from a wall) and pressure ratio
(10 .. 1e4) in water, and jittered air-helium shock-bubble set-ups.  They
exercise the band-limited work of the CUDA path (geometry after a
level-set step, fluid-1 states and Eq. 7 interpolation during sub-steps,
mixing plans) in many interface configurations: the sub-step count must
agree cycle by cycle, and the step ratio, the time and the states to
relative 1e-8 (the long-run parity bar: the most violent bubble amplifies
rounding-level differences to about 1e-9 over its ~700 fluid-2 steps)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs
from tests.test_gpu_parity import compare, sound_speed_scale

pytestmark = pytest.mark.gpu

BUBBLES = inputs.batched_instances(count=8, seed=11, nmin=40, nmax=88)


def _sif():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_03917_gb300 import sif
    return sif


def _pair(case):
    sif = _sif()
    arrs = [np.ascontiguousarray(case[x], dtype=np.float64) for x in ("phi", "prim_N", "prim_P")]
    g = sif.Solver(case["cfg"]).init_fluids(*arrs)
    o = O.Oracle(case["cfg"]).init(*arrs)
    return g, o


def _run(case, multi, n):
    g, o = _pair(case)
    for _ in range(n):
        if multi:
            a, b = g.step_multi_dt(1), o.step_multi_dt(1)
            # the same schedule: the sub-step count exactly; the used step
            # ratio, a quotient of CFL steps of states that agree to the
            # long-run parity bar, to that bar
            assert a["substeps"] == b["substeps"]
            assert abs(a["n_used"] - b["n_used"]) <= 1e-8 * b["n_used"]
        else:
            g.step_single_dt(1)
            o.step_single_dt(1)
    assert o.status == 0
    assert abs(g.t - o.t) <= 1e-8 * o.t
    return compare(g, o, 1e-8, cref=sound_speed_scale(case))


@pytest.mark.parametrize("i", range(len(BUBBLES)))
def test_bubble_instances_multi_dt(i):
    print(BUBBLES[i]["name"], "relative L1 after 60 cycles:", _run(BUBBLES[i], True, 60))


@pytest.mark.parametrize("i", [0, 3, 6])
def test_bubble_instances_single_dt(i):
    print(BUBBLES[i]["name"], "relative L1 after 60 steps:", _run(BUBBLES[i], False, 60))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_jittered_shock_bubble_multi_dt(seed):
    case = inputs.shock_bubble(128, 32, seed=seed, perturb=1e-3)
    print(case["name"], seed, "relative L1 after 120 cycles:", _run(case, True, 120))
