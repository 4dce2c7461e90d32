"""Pins of the oracle's interface Riemann solver (Sec. 2.1, interface
interaction giving the exchange flux X) against textbook values and
independent jump relations."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from tests import exact_riemann as ER

GOLD = os.path.join(os.path.dirname(__file__), "golden", "toro_ideal_gas_riemann.txt")


def _toro_rows():
    rows = []
    with open(GOLD) as f:
        lines = f.readlines()
    for line in lines:
        if line.startswith("#") or not line.strip():
            continue
        a, b = line.split("|")
        rows.append((list(map(float, a.split())), list(map(float, b.split()))))
    return rows


@pytest.mark.parametrize("row", _toro_rows())
def test_ideal_gas_star_states_match_textbook(row):
    (rl, ul, pl, rr, ur, pr), (ps, us, rsl, rsr) = row
    r = O.riemann([rl, ul, pl, 1.4, 0.0], [rr, ur, pr, 1.4, 0.0])
    assert r["rc"] == 0
    # the table prints 5-6 significant digits
    assert abs(r["p"] - ps) <= 6e-5 * abs(ps) + 1e-5
    assert abs(r["u"] - us) <= 6e-5 * abs(us) + 1e-5
    assert abs(r["rho_L"] - rsl) <= 6e-5 * rsl + 1e-5
    assert abs(r["rho_R"] - rsr) <= 6e-5 * rsr + 1e-5


WATER_AIR = ([1000.0, 0.0, 1.0e9, 4.4, 6.0e8], [1.0, 0.0, 1.0e5, 1.4, 0.0])


def test_stiffened_gas_against_independent_solver():
    L, R = WATER_AIR
    r = O.riemann(L, R)
    ps, us = ER.star_state(L, R)
    assert r["rc"] == 0 and r["iters"] < 50
    assert abs(r["p"] - ps) <= 1e-12 * ps
    assert abs(r["u"] - us) <= 1e-11 * abs(us)


def test_stiffened_gas_shock_side_satisfies_rankine_hugoniot():
    L, R = WATER_AIR
    r = O.riemann(L, R)
    rr, ur, pr, g, pi = R
    ps, us, rs = r["p"], r["u"], r["rho_R"]
    assert ps > pr  # shock into the air
    S = (rs * us - rr * ur) / (rs - rr)  # mass conservation fixes the speed
    mom_l = rr * (ur - S) ** 2 + pr
    mom_r = rs * (us - S) ** 2 + ps
    assert abs(mom_l - mom_r) <= 1e-12 * mom_l
    e = lambda p, rho: (p + g * pi) / ((g - 1.0) * rho)
    lhs = e(ps, rs) - e(pr, rr)
    rhs = 0.5 * (ps + pr) * (1.0 / rr - 1.0 / rs)
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_stiffened_gas_rarefaction_side_is_isentropic():
    L, R = WATER_AIR
    r = O.riemann(L, R)
    rl, ul, pl, g, pi = L
    ps, us, rs, cs = r["p"], r["u"], r["rho_L"], r["c_L"]
    assert ps < pl  # rarefaction into the water
    assert abs((ps + pi) / rs ** g - (pl + pi) / rl ** g) <= 1e-12 * (pl + pi) / rl ** g
    cl = math.sqrt(g * (pl + pi) / rl)
    inv_l = ul + 2.0 * cl / (g - 1.0)
    inv_s = us + 2.0 * cs / (g - 1.0)
    assert abs(inv_l - inv_s) <= 1e-12 * abs(inv_l)


def test_equal_states_give_trivial_solution():
    s = [1000.0, 3.0, 2.0e5, 4.4, 6.0e8]
    r = O.riemann(s, s)
    assert r["p"] == pytest.approx(2.0e5, rel=1e-15)
    assert r["u"] == pytest.approx(3.0, rel=1e-15)


def test_cavitation_hits_the_floor_without_failing():
    # strongly separating gas: vacuum would form; the solver floors p + p_inf
    r = O.riemann([1.0, -5000.0, 1.0e5, 1.4, 0.0], [1.0, 5000.0, 1.0e5, 1.4, 0.0])
    assert r["p"] >= 0.0 and r["p"] < 1.0
    assert np.isfinite(r["u"])
