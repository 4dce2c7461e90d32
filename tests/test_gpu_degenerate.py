"""Parity of the CUDA path with the oracle on geometries at the edges of
the cut-cell rules (Sec. 2.1, Fig. 1): zero level-set values at cell
corners on a face column, zeros at cell centres and corners on a
45-degree line (ties count as fluid P), a saddle cell with four edge
crossings, a 5 x 3 grid smaller than one finite-volume tile, and a gas
film one to two cells thick (small cells on both sides).  Both sides must
take the same discrete decisions (apertures, small-cell sources, extension
neighbours, sub-step counts) from the same input: one step or cycle to
1e-12, thirty to the long-run bar 1e-8, with the same sub-step schedule."""
import pytest

from paper_1905_03917_gb300 import inputs
from tests.test_gpu_parity import compare, pair, sound_speed_scale

pytestmark = pytest.mark.gpu

KINDS = ["face", "diagonal", "saddle", "tiny", "film"]


@pytest.mark.parametrize("kind", KINDS)
def test_single_steps(kind):
    case = inputs.degenerate(kind)
    g, o = pair(case)
    g.step_single_dt(1)
    o.step_single_dt(1)
    compare(g, o, 1e-12, cref=sound_speed_scale(case))
    g.step_single_dt(29)
    o.step_single_dt(29)
    assert o.status == 0
    assert abs(g.t - o.t) <= 1e-10 * o.t
    print(kind, "relative L1 after 30 steps:", compare(g, o, 1e-8, cref=sound_speed_scale(case)))


@pytest.mark.parametrize("kind", KINDS)
def test_multi_dt_cycles(kind):
    case = inputs.degenerate(kind)
    g, o = pair(case)
    a, b = g.step_multi_dt(1), o.step_multi_dt(1)
    assert a["substeps"] == b["substeps"]
    compare(g, o, 1e-12, cref=sound_speed_scale(case))
    for _ in range(29):
        a, b = g.step_multi_dt(1), o.step_multi_dt(1)
        assert a["substeps"] == b["substeps"]
    assert o.status == 0
    assert abs(g.t - o.t) <= 1e-10 * o.t
    print(kind, "relative L1 after 30 cycles:", compare(g, o, 1e-8, cref=sound_speed_scale(case)))
