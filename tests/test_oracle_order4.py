"""Pins of the optional fourth-order D2Q9 term (H_xxyy, reading R23).

  * Hermite facts: H_xxyy is orthogonal on D2Q9 to every polynomial the
    order-3 expansion uses, with the continuous norm 4 c_s^8
  * the order-4 equilibrium carries the Maxwell-Boltzmann fourth moment
    rho u_x^2 u_y^2 on H_xxyy, the order-3 one carries none
  * Eq. recursive2 at n = 4 (symmetric sum over index pairs), evaluated by
    hand: a4_xxyy = u_x^2 P_yy + u_y^2 P_xx + 4 u_x u_y P_xy
  * collision invariants, projector, tau = 1, and the order-4 collision
    changes only the H_xxyy component of the rebuilt populations
"""
import numpy as np
import pytest

import oracle
from oracle import CS2, D2Q9


def _lat():
    d, q, xi, w, opp = oracle.lattice(D2Q9)
    return xi.astype(float), w


def _h4(xi):
    return (xi[:, 0] ** 2 - CS2) * (xi[:, 1] ** 2 - CS2)


def _one_cell(tau, order4):
    P = oracle.Problem(D2Q9, (1, 1), tau)
    P.order4 = order4
    return P


def test_h_xxyy_is_orthogonal_with_the_continuous_norm():
    xi, w = _lat()
    h4 = _h4(xi)
    lower = [np.ones(9), xi[:, 0], xi[:, 1], xi[:, 0] ** 2 - CS2, xi[:, 0] * xi[:, 1], xi[:, 1] ** 2 - CS2,
             (xi[:, 0] ** 2 - CS2) * xi[:, 1], (xi[:, 1] ** 2 - CS2) * xi[:, 0]]
    for p in lower:
        assert abs((w * h4 * p).sum()) < 1e-16
    assert abs((w * h4 * h4).sum() - 4 * CS2 ** 4) < 1e-16


def test_order4_equilibrium_carries_the_maxwell_fourth_moment():
    xi, w = _lat()
    rng = np.random.default_rng(4)
    for _ in range(6):
        rho, u = 0.9 + 0.2 * rng.random(), np.append(0.2 * rng.normal(size=2), 0.0)
        f4 = _one_cell(1.0, 1).equilibrium(np.array([rho]), u[None, :])[:, 0]
        f3 = _one_cell(1.0, 0).equilibrium(np.array([rho]), u[None, :])[:, 0]
        assert abs((f4 * _h4(xi)).sum() - rho * u[0] ** 2 * u[1] ** 2) < 1e-16
        assert abs((f3 * _h4(xi)).sum()) < 1e-16
        # the two differ exactly by the H_xxyy term
        assert np.abs(f4 - f3 - w * _h4(xi) * rho * u[0] ** 2 * u[1] ** 2 / (4 * CS2 ** 4)).max() < 1e-16


def test_recursive_fourth_order_special_case():
    """Regularized populations (tau -> infinity) rebuilt from a state with
    given u and Pi^neq carry a4_xxyy on H_xxyy."""
    xi, w = _lat()
    rng = np.random.default_rng(5)
    for _ in range(5):
        f = w * (1 + 0.2 * (2 * rng.random(9) - 1))
        rho = f.sum()
        u = (f[:, None] * xi).sum(0) / rho
        Pi = np.einsum("i,ia,ib->ab", f, xi, xi)
        pn = Pi - rho * CS2 * np.eye(3) - rho * np.outer(u, u)
        reg = oracle.collide(D2Q9, f, 1e300, order4=True)
        want = rho * u[0] ** 2 * u[1] ** 2 + u[0] ** 2 * pn[1, 1] + u[1] ** 2 * pn[0, 0] + 4 * u[0] * u[1] * pn[0, 1]
        assert abs((reg * _h4(xi)).sum() - want) < 1e-15


@pytest.mark.parametrize("tau", [0.53, 0.8, 1.0, 1.6])
def test_order4_collision_conserves_and_projects(tau):
    xi, w = _lat()
    rng = np.random.default_rng(6)
    for _ in range(5):
        f = w * (1 + 0.3 * (2 * rng.random(9) - 1))
        out = oracle.collide(D2Q9, f, tau, order4=True)
        assert abs(out.sum() - f.sum()) < 1e-15
        assert np.abs((out[:, None] * xi).sum(0) - (f[:, None] * xi).sum(0)).max() < 1e-15
        reg = oracle.collide(D2Q9, f, 1e300, order4=True)
        assert np.abs(oracle.collide(D2Q9, reg, 1e300, order4=True) - reg).max() < 1e-15
        # order 3 and order 4 differ only along H_xxyy
        d = out - oracle.collide(D2Q9, f, tau, order4=False)
        assert np.abs(d - w * _h4(xi) * (d * _h4(xi)).sum() / (4 * CS2 ** 4)).max() < 1e-15
    f = w * (1 + 0.1 * rng.random(9))
    rho = f.sum()
    u = np.append((f[:, None] * xi).sum(0)[:2] / rho, 0.0)
    feq = _one_cell(1.0, 1).equilibrium(np.array([rho]), u[None, :])[:, 0]
    assert np.abs(oracle.collide(D2Q9, f, 1.0, order4=True) - feq).max() < 1e-15
