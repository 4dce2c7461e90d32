"""Pins of the oracle on geometries at the edges of the cut-cell rules
(Sec. 2.1, Fig. 1): an interface exactly on a column of cell faces, a
45-degree interface through cell centres and corners, a saddle cell with
four edge crossings, a grid smaller than one tile, and a gas film one to
two cells thick.  What the method fixes there whatever the implementation:
each fluid's mass and the total energy are conserved in a reflective box
(the interfacial exchange carries no mass and is antisymmetric between the
fluids; walls do no work), a planar interface on a face column stays
planar with no transverse momentum, and the 45-degree case keeps its
reflection symmetry (x, y) -> (1 - y, 1 - x)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs

KINDS = ["face", "diagonal", "saddle", "tiny", "film"]


def _run(kind, multi, n):
    c = inputs.degenerate(kind)
    o = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    I0 = o.integrals()
    subs = []
    for _ in range(n):
        if multi:
            subs.append(o.step_multi_dt(1)["substeps"])
        else:
            o.step_single_dt(1)
    assert o.status == 0
    return o, I0, subs


def test_inputs_reach_the_degenerate_rules():
    # exact zeros at centres (ties) and corners for the diagonal; zero
    # corner values on the face column; alternating corner signs around
    # the saddle point; a gas pocket the tiny grid's geometry sees
    d = inputs.degenerate("diagonal")["phi"]
    assert (d == 0).sum() == d.shape[0]
    corners = lambda p: 0.25 * (p[:-1, :-1] + p[1:, :-1] + p[:-1, 1:] + p[1:, 1:])
    f = corners(inputs.degenerate("face")["phi"])
    assert (f == 0).any()
    s = corners(inputs.degenerate("saddle")["phi"]) >= 0
    alt = (s[:-1, :-1] == s[1:, 1:]) & (s[1:, :-1] == s[:-1, 1:]) & (s[:-1, :-1] != s[1:, :-1])
    assert alt.any()
    c = inputs.degenerate("tiny")
    o = O.Oracle(c["cfg"]).init(c["phi"], c["prim_N"], c["prim_P"])
    assert o.integrals()[0, 0] > 0


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("multi", [False, True])
def test_mass_of_each_fluid_and_total_energy_are_conserved(kind, multi):
    o, I0, subs = _run(kind, multi, 30)
    I1 = o.integrals()
    for k in range(2):
        assert abs(I1[k, 0] - I0[k, 0]) <= 1e-13 * abs(I0[k, 0])
    E0, E1 = I0[:, 3].sum(), I1[:, 3].sum()
    assert abs(E1 - E0) <= 1e-13 * abs(E0)
    if multi and kind in ("face", "diagonal", "saddle", "film"):
        assert max(subs) >= 3  # the water's steps are sub-cycled


@pytest.mark.parametrize("multi", [False, True])
def test_interface_on_a_face_column_stays_planar(multi):
    o, _, _ = _run("face", multi, 30)
    qN, qP, phi = o.state()
    for q in (qN, qP):
        for m in range(4):
            assert np.array_equal(q[m], np.broadcast_to(q[m][0], q[m].shape))
        assert not q[2].any()
    assert np.array_equal(phi, np.broadcast_to(phi[0], phi.shape))
    assert np.abs(qP[1]).max() > 0  # the water has pushed the gas


@pytest.mark.parametrize("multi", [False, True])
def test_diagonal_interface_keeps_its_reflection_symmetry(multi):
    o, _, _ = _run("diagonal", multi, 30)
    qN, qP, phi = o.state()
    T = lambda a: a[::-1, ::-1].T  # value at the image of (x, y) under (1 - y, 1 - x)
    for q in (qN, qP):
        for m in (0, 3):
            assert np.abs(q[m] - T(q[m])).max() <= 1e-11 * np.abs(q[m]).max()
        scale = np.abs(q[1]).max()
        assert scale > 0
        # the reflection maps velocity (u, v) to (-v, -u)
        assert np.abs(q[1] + T(q[2])).max() <= 1e-8 * scale
    assert np.abs(phi - T(phi)).max() <= 1e-12
