"""Host-side arithmetic of the benchmark's multi- vs single-time-step
comparison: the conservative 2 x 2 average onto the coarse grid and the
speedup model of Eq. 13."""
import numpy as np

import bench


def test_coarsening_conserves_and_averages():
    rng = np.random.default_rng(3)
    a = rng.random((2, 6, 10))
    c = bench._coarsen(a)
    assert c.shape == (2, 3, 5)
    assert np.isclose(c.sum() * 4, a.sum())
    assert np.isclose(c[1, 2, 4], a[1, 4:6, 8:10].mean())


def test_eq13_limits_and_the_papers_example():
    # fluid 1 takes all the time: the speedup is the time-step ratio n
    assert bench._eq13(2.8, 3, 1.0) == 2.8
    # fluid 1 takes none of it: [n] fluid-2 steps cover n single steps
    assert np.isclose(bench._eq13(2.8, 3, 0.0), 2.8 / 3)
    # Sec. 3.1's example (dt1 = 2.8 dt2): three fluid-2 steps and one
    # fluid-1 step advance as far as 2.8 single steps; with fluid 1 at
    # 3/4 of a step's time the cycle costs 3 - 2 x 0.75 = 1.5 steps
    assert np.isclose(bench._eq13(2.8, 3, 0.75), 2.8 / 1.5)
    # integer ratio with one sub-step: the original method
    assert bench._eq13(1.0, 1, 0.3) == 1.0


def test_time_at_error_interpolates_log_log_and_never_extrapolates():
    curve = [{"cfl": 0.6, "err": 4e-3, "ms": 100.0}, {"cfl": 0.3, "err": 1e-3, "ms": 200.0}]
    # halfway in log error is halfway in log time
    assert np.isclose(bench._time_at_error(curve, 2e-3), 100.0 * np.sqrt(2.0))
    assert bench._time_at_error(curve, 4e-3) == 100.0
    assert bench._time_at_error(curve, 1e-3) == 200.0
    assert bench._time_at_error(curve, 5e-3) is None
    assert bench._time_at_error(curve, 5e-4) is None


def test_equal_error_speedup_takes_the_looser_common_error():
    single = [{"cfl": 0.6, "err": 2e-3, "ms": 100.0}, {"cfl": 0.3, "err": 5e-4, "ms": 200.0}]
    # multi-step: larger error at the same CFL number, half the time
    multi = [{"cfl": 0.6, "err": 4e-3, "ms": 50.0}, {"cfl": 0.3, "err": 1e-3, "ms": 100.0}]
    sp, e_star, curve = bench.equal_error_speedup(single, multi)
    assert e_star == 2e-3
    # multi needs 50 * sqrt(2) ms for 2e-3 (halfway in log error)
    assert np.isclose(sp, 100.0 / (50.0 * np.sqrt(2.0)))
    assert np.isclose(curve[0]["speedup"], sp)
    assert curve[1]["speedup"] is None          # 5e-4 lies outside the multi sweep
    # the other way round: multi more accurate at CFL 0.6
    sp2, e2, _ = bench.equal_error_speedup(multi, single)
    assert e2 == 2e-3 and np.isclose(sp2, 50.0 * np.sqrt(2.0) / 100.0)


def test_partition_covers_every_instance_once():
    for n in (1, 7, 256):
        for ws in (1, 2, 3, 8):
            parts = [bench.partition(n, r, ws) for r in range(ws)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
