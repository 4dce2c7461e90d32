"""Batched instances (many independent problems of uneven grid sizes, one
graph launch per batch cycle) and the tile-shape autotuner: every instance
of a batch equals the same instance advanced alone, bitwise, and results
do not depend on the finite-volume tile shape."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs
from tests.test_gpu_parity import compare, sound_speed_scale

pytestmark = pytest.mark.gpu


def _sif():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_03917_gb300 import sif
    return sif


def _arrays(case):
    return [np.ascontiguousarray(case[x]) for x in ("phi", "prim_N", "prim_P")]


def test_batch_instances_equal_solo_runs_bitwise():
    sif = _sif()
    cases = inputs.batched_instances(count=6, seed=3, nmin=40, nmax=96)
    b = sif.Batch([c["cfg"] for c in cases])
    for s, c in zip(b.instances, cases):
        s.init_fluids(*_arrays(c))
    upd = b.step_multi_dt(4)
    assert upd > 0
    for s, c in zip(b.instances, cases):
        solo = sif.Solver(c["cfg"]).init_fluids(*_arrays(c))
        solo.step_multi_dt(4)
        for x, y in zip(s.state(), solo.state()):
            assert np.array_equal(x, y)
        assert s.t == solo.t


def test_batch_instance_matches_oracle():
    sif = _sif()
    cases = inputs.batched_instances(count=3, seed=5, nmin=40, nmax=72)
    b = sif.Batch([c["cfg"] for c in cases])
    for s, c in zip(b.instances, cases):
        s.init_fluids(*_arrays(c))
    b.step_multi_dt(3)
    for s, c in zip(b.instances, cases):
        o = O.Oracle(c["cfg"]).init(*_arrays(c))
        o.step_multi_dt(3)
        compare(s, o, 1e-12, cref=sound_speed_scale(c))


@pytest.mark.parametrize("shape", [(32, 4), (16, 8), (16, 16), (64, 4)])
def test_results_do_not_depend_on_tile_shape(shape):
    sif = _sif()
    case = inputs.underwater_explosion(77, radius=0.3, p_gas=1e8, rho_gas=1.0, seed=7)
    a = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    b = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    b.set_tile_shape(*shape)
    assert b.tile_shape == shape
    a.step_multi_dt(3)
    b.step_multi_dt(3)
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)


def test_autotuner_picks_a_shape_and_restores_state(tmp_path):
    sif = _sif()
    from paper_1905_03917_gb300 import autotune
    case = inputs.underwater_explosion(96, radius=0.3, p_gas=1e8, rho_gas=1.0, seed=2)
    s = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    before = [x.copy() for x in s.state()]
    shape, rec = autotune.tune(s, cache=str(tmp_path / "tune.json"))
    assert tuple(shape) in autotune.SHAPES
    assert s.tile_shape == tuple(shape)
    for x, y in zip(before, s.state()):
        assert np.array_equal(x, y)
    assert all(v > 0 for v in rec["ms_per_cycle"].values())
    again, _ = autotune.tune(s, cache=str(tmp_path / "tune.json"))
    assert tuple(again) == tuple(shape)


def test_unsupported_tile_shape_is_rejected():
    sif = _sif()
    case = inputs.static_interface(32, 32)
    s = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    with pytest.raises(sif.SifError) as e:
        s.set_tile_shape(24, 8)
    assert e.value.code == sif.EINVAL
