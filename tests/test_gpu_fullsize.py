"""Parity at the full sizes of the measured workloads, in the launch
configuration the benchmark times: tile shape from the autotuner, graph
launches, one call per cycle after warm-up cycles.

* the air-helium shock-bubble interaction on 1024 x 256 (Sec. 4.2),
  multi-time-step cycles against the oracle, relative L1 <= 1e-12;
* the underwater explosion on 2048 x 2048 (Sec. 4.1), one cycle against
  the oracle at the same bar, plus conservation of the totals;
* the batch of 256 independent gas-water instances (64^2 .. 512^2), one
  graph launch per batch cycle: every instance bitwise equal to the same
  instance advanced alone, and seeded samples against the oracle;
* the shock-bubble with the characteristic reconstruction and with the
  HLLC face flux, three cycles each against the oracle;
* the translating Tait droplet (the paper's Table 1 case) at 256^2, four
  cycles against the oracle."""
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
    return [np.ascontiguousarray(case[x], dtype=np.float64) for x in ("phi", "prim_N", "prim_P")]


def _oracle(case):
    o = O.Oracle(case["cfg"]).init(case["phi"], case["prim_N"], case["prim_P"])
    o.cref = sound_speed_scale(case)
    return o


def test_shock_bubble_1024x256_bench_configuration(tmp_path):
    sif = _sif()
    from paper_1905_03917_gb300 import autotune
    case = inputs.shock_bubble(1024, 256)
    s = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    shape, _ = autotune.tune(s, cache=str(tmp_path / "tune.json"), cycles=2)
    assert s.t == 0.0  # tuning leaves the initial state in place
    infos = [s.step_multi_dt(1) for _ in range(5)]
    o = _oracle(case)
    oinfos = [o.step_multi_dt(1) for _ in range(5)]
    for a, b in zip(infos, oinfos):
        assert a["substeps"] == b["substeps"] and a["n_used"] == b["n_used"]
        assert abs(a["t"] - b["t"]) <= 1e-13 * b["t"]
    assert o.status == 0
    worst = compare(s, o, 1e-12)
    print("tile", shape, "relative L1 after 5 cycles:", worst)


def test_underwater_explosion_2048_one_cycle():
    sif = _sif()
    case = inputs.underwater_explosion(2048)
    s = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    before = s.integrals()
    s.step_multi_dt(1)
    after = s.integrals()
    o = _oracle(case)
    o.step_multi_dt(1)
    assert o.status == 0
    assert abs(s.t - o.t) <= 1e-13 * o.t
    worst = compare(s, o, 1e-12)
    print("relative L1 after one cycle:", worst)
    # reflective walls: mass and energy of the mixture are conserved to
    # round-off (Eq. 8-9 keep the correction conservative)
    for m in (0, 3):
        tot0 = before[0][m] + before[1][m]
        tot1 = after[0][m] + after[1][m]
        assert abs(tot1 - tot0) <= 1e-12 * abs(tot0), (m, tot0, tot1)


def test_batch_of_256_instances(tmp_path):
    sif = _sif()
    from paper_1905_03917_gb300 import autotune
    cases = inputs.batched_instances(count=256, seed=0)
    b = sif.Batch([c["cfg"] for c in cases])
    for s, c in zip(b.instances, cases):
        s.init_fluids(*_arrays(c))
    autotune.tune_batch(b, cache=str(tmp_path / "tune.json"), cycles=1)
    ncyc = 3
    for _ in range(ncyc):
        assert b.step_multi_dt(1) > 0
    for s, c in zip(b.instances, cases):
        solo = sif.Solver(c["cfg"]).init_fluids(*_arrays(c))
        solo.step_multi_dt(ncyc)
        for x, y in zip(s.state(), solo.state()):
            assert np.array_equal(x, y), c["name"]
        assert s.t == solo.t
        solo.close()
    # seeded sample against the oracle: the smallest and the largest grids
    # and a few others
    sizes = [c["cfg"]["nx"] for c in cases]
    rng = np.random.default_rng(17)
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes))}
    pick |= {int(i) for i in rng.choice(len(cases), size=3, replace=False)}
    for i in sorted(pick):
        o = _oracle(cases[i])
        o.step_multi_dt(ncyc)
        assert o.status == 0
        compare(b.instances[i], o, 1e-12)


def test_shock_bubble_1024x256_characteristic(tmp_path):
    """The characteristic-wise option at the same size and in the same launch
    configuration (`bench.py --weno characteristic`): graph launches, tile
    shape from the autotuner, three cycles against the oracle."""
    sif = _sif()
    from paper_1905_03917_gb300 import autotune
    case = inputs.shock_bubble(1024, 256)
    case["cfg"] = dict(case["cfg"], weno_char=1)
    s = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    shape, _ = autotune.tune(s, cache=str(tmp_path / "tune.json"), cycles=2)
    infos = [s.step_multi_dt(1) for _ in range(3)]
    o = _oracle(case)
    oinfos = [o.step_multi_dt(1) for _ in range(3)]
    for a, b in zip(infos, oinfos):
        assert a["substeps"] == b["substeps"] and a["n_used"] == b["n_used"]
        assert abs(a["t"] - b["t"]) <= 1e-13 * b["t"]
    assert o.status == 0
    print("tile", shape, "relative L1 after 3 cycles:", compare(s, o, 1e-12))


def test_shock_bubble_1024x256_hllc(tmp_path):
    """The HLLC face flux at the same size and in the same launch
    configuration (`bench.py --flux hllc`): graph launches, tile shape from
    the autotuner, three cycles against the oracle."""
    sif = _sif()
    from paper_1905_03917_gb300 import autotune
    case = inputs.shock_bubble(1024, 256)
    case["cfg"] = dict(case["cfg"], flux="hllc")
    s = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    shape, _ = autotune.tune(s, cache=str(tmp_path / "tune.json"), cycles=2)
    infos = [s.step_multi_dt(1) for _ in range(3)]
    o = _oracle(case)
    oinfos = [o.step_multi_dt(1) for _ in range(3)]
    for a, b in zip(infos, oinfos):
        assert a["substeps"] == b["substeps"] and a["n_used"] == b["n_used"]
        assert abs(a["t"] - b["t"]) <= 1e-13 * b["t"]
        assert a["open_updates"] == b["open_updates"]
    assert o.status == 0
    print("tile", shape, "relative L1 after 3 cycles:", compare(s, o, 1e-12))


def test_droplet_translation_256_bench_configuration(tmp_path):
    """The paper's Table 1 case (Tait water in air, periodic) at 256^2 in the
    launch configuration `bench.py --workload paper_table1` times: graph
    launches, tile shape from the autotuner, four accelerated cycles of
    about four water sub-steps against the oracle."""
    sif = _sif()
    from paper_1905_03917_gb300 import autotune
    case = inputs.droplet_translation(256)
    s = sif.Solver(case["cfg"]).init_fluids(*_arrays(case))
    shape, _ = autotune.tune(s, cache=str(tmp_path / "tune.json"), cycles=2)
    infos = [s.step_multi_dt(1) for _ in range(4)]
    o = _oracle(case)
    oinfos = [o.step_multi_dt(1) for _ in range(4)]
    for a, b in zip(infos, oinfos):
        assert a["substeps"] == b["substeps"] >= 3
        assert abs(a["t"] - b["t"]) <= 1e-13 * b["t"]
        assert a["open_updates"] == b["open_updates"]
    assert o.status == 0
    print("tile", shape, "relative L1 after 4 cycles:", compare(s, o, 1e-12))
