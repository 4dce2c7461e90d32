"""The physics options together and inside the batched graph: the
shock-bubble with characteristic-wise WENO5 (or the HLLC face flux),
surface tension and viscosity at once against the oracle (one cycle to
1e-12, twenty to 1e-8 with the same schedule), and a batch whose instances
use different options equal to the same instances advanced alone,
bitwise."""
import numpy as np
import pytest

from paper_1905_03917_gb300 import inputs
from tests.test_gpu_parity import compare, pair, sound_speed_scale

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("flux", [{"weno_char": 1}, {"flux": "hllc"}])
def test_all_options_together_against_the_oracle(flux):
    case = inputs.shock_bubble(128, 32, seed=3, perturb=1e-3)
    case["cfg"] = dict(case["cfg"], sigma=0.02, mu=(2e-4, 1e-4), **flux)
    cref = sound_speed_scale(case)
    g, o = pair(case)
    a, b = g.step_multi_dt(1), o.step_multi_dt(1)
    assert a["substeps"] == b["substeps"]
    compare(g, o, 1e-12, cref=cref)
    for _ in range(19):
        a, b = g.step_multi_dt(1), o.step_multi_dt(1)
        assert a["substeps"] == b["substeps"]
    assert o.status == 0
    print("relative L1 after 20 cycles:", compare(g, o, 1e-8, cref=cref))


def test_batch_with_options_equals_solo_runs_bitwise():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_03917_gb300 import sif
    cases = inputs.batched_instances(count=5, seed=9, nmin=40, nmax=72)
    opts = [{}, {"weno_char": 1}, {"sigma": 1.0e3}, {"mu": (5.0e-2, 1.0e-3)}, {"flux": "hllc"}]
    for c, extra in zip(cases, opts):
        c["cfg"] = dict(c["cfg"], **extra)
    arrs = lambda c: [np.ascontiguousarray(c[x]) for x in ("phi", "prim_N", "prim_P")]
    b = sif.Batch([c["cfg"] for c in cases])
    for s, c in zip(b.instances, cases):
        s.init_fluids(*arrs(c))
    b.step_multi_dt(3)
    for s, c in zip(b.instances, cases):
        solo = sif.Solver(c["cfg"]).init_fluids(*arrs(c))
        solo.step_multi_dt(3)
        for x, y in zip(s.state(), solo.state()):
            assert np.array_equal(x, y)
        assert s.t == solo.t
