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
