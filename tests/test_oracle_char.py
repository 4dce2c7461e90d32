"""Pins of the oracle's characteristic-wise WENO5 option (a reconstruction
the paper does not use; its WENO-LF of Sec. 4 is component-wise): the
eigenvector basis against the Euler equations themselves, and the scheme
built on it against the properties any consistent, conservative
fifth-order scheme has.

* The right eigenvectors diagonalise the flux Jacobian dF/dU, with the
  Jacobian taken by complex-step differentiation of the Euler flux of a
  stiffened gas written out here (not the oracle's formulas), to eigenvalues
  un - c, un, un, un + c; the left eigenvectors are their inverse.
* The single-fluid operator stays fifth order on smooth data.
* The water-air shock tube converges to the exact solution.
* The multi-time-step cycle with the flux correction conserves mass,
  momentum and energy."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_03917_gb300 import inputs
from tests.test_oracle_physics import _drift, _tube_errors
from tests.test_oracle_scheme import _exact_divergence, _smooth_single_fluid


def _euler_flux(U, d, g, pinf):
    rho, mx, my, E = U
    u, v = mx / rho, my / rho
    p = (g - 1.0) * (E - 0.5 * rho * (u * u + v * v)) - g * pinf
    un = u if d == 0 else v
    return np.array([rho * un, mx * un + (p if d == 0 else 0.0),
                     my * un + (p if d == 1 else 0.0), un * (E + p)])


def _jacobian(U, d, g, pinf):
    A = np.empty((4, 4))
    for j in range(4):
        h = 1e-20 * max(abs(U[j]), 1.0)
        Uc = U.astype(complex)
        Uc[j] += 1j * h
        A[:, j] = _euler_flux(Uc, d, g, pinf).imag / h
    return A


STATES = [(1.4, 0.0, 1.2, 30.0, -20.0, 1.0e5), (1.4, 0.0, 0.138, 0.0, 0.0, 1.0),
          (4.4, 6.0e8, 1000.0, 3.0, 2.0, 1.0e6), (4.4, 6.0e8, 1020.0, -150.0, 40.0, 1.0e9),
          (1.67, 0.0, 0.2, -0.5, 0.9, 2.0)]


@pytest.mark.parametrize("state", STATES)
@pytest.mark.parametrize("d", [0, 1])
def test_basis_diagonalises_the_flux_jacobian(state, d):
    g, pinf, rho, u, v, p = state
    L, R = O.char_basis(g, pinf, rho, u, v, p, d)
    E = (p + g * pinf) / (g - 1.0) + 0.5 * rho * (u * u + v * v)
    U = np.array([rho, rho * u, rho * v, E])
    A = _jacobian(U, d, g, pinf)
    un = u if d == 0 else v
    c = np.sqrt(g * (p + pinf) / rho)
    lam = np.array([un - c, un, un, un + c])
    # A r_f = lambda_f r_f, column by column on each column's own scale
    for f in range(4):
        res = A @ R[:, f] - lam[f] * R[:, f]
        scale = np.abs(A).max(axis=1) @ np.abs(R[:, f]) + abs(lam[f]) * np.abs(R[:, f]).max()
        assert np.abs(res).max() <= 1e-13 * scale, (f, res)
    # L = R^-1: L R = I and R L = I (relative to the entries' products)
    assert np.abs(L @ R - np.eye(4)).max() <= 1e-13 * (np.abs(L) @ np.abs(R)).max()
    assert np.abs(R @ L - np.eye(4)).max() <= 1e-13 * (np.abs(R) @ np.abs(L)).max()
    # the four fields are distinct waves: the basis is not degenerate
    assert abs(np.linalg.det(R)) > 0


def test_basis_rejects_a_non_physical_state():
    with pytest.raises(ValueError):
        O.char_basis(4.4, 6.0e8, 1000.0, 0.0, 0.0, -7.0e8, 0)


def test_characteristic_operator_is_fifth_order():
    errs = []
    for n in (16, 32, 64):
        cfg, X, Y, phi, pr = _smooth_single_fluid(n)
        cfg["weno_char"] = 1
        o = O.Oracle(cfg).init(phi, pr, pr)
        errs.append(np.abs(o.rhs(1) - _exact_divergence(X, Y)).max())
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 4.5, (errs, orders)


@pytest.mark.parametrize("multi", [False, True])
def test_characteristic_shock_tube_converges(multi):
    errs, cons = zip(*(_tube_errors(n, 2, multi, weno_char=1) for n in (200, 400, 800)))
    assert all(b < 0.8 * a for a, b in zip(errs, errs[1:])), errs
    assert max(cons) <= 2.0, cons


def test_characteristic_multi_dt_conserves():
    c = inputs.periodic_bubble(48, seed=1)
    cfg = dict(c["cfg"], weno_char=1)
    o = O.Oracle(cfg).init(c["phi"], c["prim_N"], c["prim_P"])
    I0 = o.integrals().sum(0)
    subs = [o.step_multi_dt(1)["substeps"] for _ in range(40)]
    assert o.status == 0 and max(subs) >= 2
    assert _drift(o, I0).max() <= 1e-13


def test_characteristic_and_componentwise_agree_on_smooth_data():
    # both are fifth-order approximations of the same divergence: on a
    # smooth field their difference shrinks at that order too
    diffs = []
    for n in (16, 32, 64):
        cfg, X, Y, phi, pr = _smooth_single_fluid(n)
        a = O.Oracle(cfg).init(phi, pr, pr).rhs(1)
        b = O.Oracle(dict(cfg, weno_char=1)).init(phi, pr, pr).rhs(1)
        diffs.append(np.abs(a - b).max())
    assert diffs[0] > 0
    assert all(np.log2(diffs[i] / diffs[i + 1]) >= 4.0 for i in range(2)), diffs


def test_the_two_reconstructions_differ_by_more_than_the_parity_bar():
    # so that agreement of the CUDA path with the oracle at 1e-12 in this
    # mode shows that it took the characteristic path
    case = inputs.shock_bubble(128, 32, seed=3, perturb=1e-3)
    a = O.Oracle(case["cfg"]).init(case["phi"], case["prim_N"], case["prim_P"])
    b = O.Oracle(dict(case["cfg"], weno_char=1)).init(case["phi"], case["prim_N"], case["prim_P"])
    a.step_single_dt(1)
    b.step_single_dt(1)
    qa, qb = a.state()[1], b.state()[1]
    assert np.abs(qa - qb).sum() / np.abs(qa).sum() > 1e-9
