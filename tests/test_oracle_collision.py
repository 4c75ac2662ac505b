"""Pins of the oracle's lattice tables and single-cell collision.

Every expected value here comes from mathematics the paper fixes, not from the
oracle itself: quadrature identities of the lattices, conservation of mass and
momentum by Eq. optimizedLB, the continuous Maxwell-Boltzmann moments that the
third-order equilibrium (Eq. eqH) must reproduce, hand-evaluated special cases
of the recursion Eq. recursive2, and closed forms of the sponge update
(Eq. spongeLB, Eq. dampingLBM) in a homogeneous cell.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from oracle import D2Q9, D3Q19, D3Q27, CS2

LATS = [D2Q9, D3Q19, D3Q27]
Q = {D2Q9: 9, D3Q19: 19, D3Q27: 27}


def _lat(which):
    d, q, xi, w, opp = oracle.lattice(which)
    return d, q, xi.astype(np.float64), w, opp


@pytest.mark.parametrize("which", LATS)
def test_lattice_quadrature_identities(which):
    """Sum w = 1, odd moments vanish, sum w xi xi = c_s^2 I, 4th-order isotropy."""
    d, q, xi, w, opp = _lat(which)
    assert q == Q[which]
    assert abs(w.sum() - 1.0) < 1e-15
    for a in range(3):
        assert abs((w * xi[:, a]).sum()) < 1e-15
    for a, b in itertools.product(range(d), repeat=2):
        assert abs((w * xi[:, a] * xi[:, b]).sum() - CS2 * (a == b)) < 1e-15
    for a, b, c in itertools.product(range(d), repeat=3):
        assert abs((w * xi[:, a] * xi[:, b] * xi[:, c]).sum()) < 1e-15
    dl = lambda i, j: 1.0 if i == j else 0.0
    for a, b, c, e in itertools.product(range(d), repeat=4):
        want = CS2 ** 2 * (dl(a, b) * dl(c, e) + dl(a, c) * dl(b, e) + dl(a, e) * dl(b, c))
        assert abs((w * xi[:, a] * xi[:, b] * xi[:, c] * xi[:, e]).sum() - want) < 1e-15
    if which == D3Q27:
        # the tensor-product lattice: weights factor into D1Q3 weights (2/3, 1/6, 1/6)
        w1 = {0: 2 / 3, 1: 1 / 6, -1: 1 / 6}
        for i in range(q):
            v = xi[i].astype(int)
            assert abs(w[i] - w1[v[0]] * w1[v[1]] * w1[v[2]]) < 1e-16


@pytest.mark.parametrize("which", LATS)
def test_lattice_opposites_and_order(which):
    d, q, xi, w, opp = _lat(which)
    h = q // 2
    assert np.all(xi[0] == 0)
    for i in range(q):
        assert np.all(xi[opp[i]] == -xi[i])
    for i in range(1, h + 1):
        assert opp[i] == i + h
    # all velocities distinct, unit components only; corner velocities only on D3Q27
    assert len({tuple(v) for v in xi.astype(int)}) == q
    assert np.abs(xi).max() == 1
    assert (np.abs(xi).sum(axis=1) <= (3 if which == D3Q27 else 2)).all()
    if which == D2Q9:
        assert np.all(xi[:, 2] == 0)


def _random_f(which, seed, spread=0.3):
    d, q, xi, w, opp = _lat(which)
    rng = np.random.default_rng(seed)
    f = w * (1.0 + spread * (2 * rng.random(q) - 1))
    # add a mean flow so that third-order terms are active
    f = f * (1 + 0.2 * (xi @ rng.normal(size=3)) * (rng.random() - 0.5))
    return np.abs(f)


def _moments(which, f):
    d, q, xi, w, opp = _lat(which)
    rho = f.sum()
    j = (f[:, None] * xi).sum(axis=0)
    Pi = np.einsum("i,ia,ib->ab", f, xi, xi)
    return rho, j, Pi


@pytest.mark.parametrize("which", LATS)
@pytest.mark.parametrize("tau", [0.51, 0.6, 1.0, 1.7])
def test_collision_conserves_mass_and_momentum(which, tau):
    for seed in range(20):
        f = _random_f(which, seed)
        out = oracle.collide(which, f, tau)
        r0, j0, _ = _moments(which, f)
        r1, j1, _ = _moments(which, out)
        assert abs(r1 - r0) <= 1e-14 * r0
        assert np.abs(j1 - j0).max() <= 1e-14 * r0


@pytest.mark.parametrize("which", LATS)
def test_regularized_populations_reproduce_second_moment(which):
    """feqH + fneqH rebuilt from (rho, u, Pi^neq) has the input's rho, j, Pi."""
    for seed in range(10):
        f = _random_f(which, seed)
        rho, j, Pi = _moments(which, f)
        u = j / rho
        pn = Pi - rho * CS2 * np.eye(3) - rho * np.outer(u, u)
        freg = oracle.feqH(which, rho, u) + oracle.fneqH(which, u, pn)
        r1, j1, P1 = _moments(which, freg)
        assert abs(r1 - rho) < 1e-14
        assert np.abs(j1 - j).max() < 1e-14
        d = 2 if which == D2Q9 else 3
        assert np.abs(P1[:d, :d] - Pi[:d, :d]).max() < 1e-14


@pytest.mark.parametrize("which", LATS)
def test_regularization_is_a_projector(which):
    """Collision with tau -> infinity returns the regularized f; applying it twice changes nothing."""
    for seed in range(5):
        f = _random_f(which, seed)
        r1 = oracle.collide(which, f, 1e300)
        r2 = oracle.collide(which, r1, 1e300)
        assert np.abs(r2 - r1).max() < 1e-15


@pytest.mark.parametrize("which", LATS)
def test_tau_one_gives_equilibrium_and_equilibrium_is_fixed(which):
    for seed in range(5):
        f = _random_f(which, seed)
        rho, j, _ = _moments(which, f)
        feq = oracle.feqH(which, rho, j / rho)
        assert np.abs(oracle.collide(which, f, 1.0) - feq).max() < 1e-15
        assert np.abs(oracle.collide(which, feq, 0.7) - feq).max() < 1e-15


@pytest.mark.parametrize("which", LATS)
def test_equilibrium_matches_textbook_second_order_for_axis_aligned_flow(which):
    """For u along one axis every supported third-order term vanishes, so
    Eq. eqH must equal the quadratic equilibrium Eq. truncatedEq exactly."""
    d, q, xi, w, opp = _lat(which)
    for axis in range(d):
        for U in (0.05, -0.17):
            u = np.zeros(3)
            u[axis] = U
            rho = 1.03
            xu = xi @ u
            textbook = w * rho * (1 + xu / CS2 + xu ** 2 / (2 * CS2 ** 2) - (u @ u) / (2 * CS2))
            assert np.abs(oracle.feqH(which, rho, u) - textbook).max() < 1e-16


@pytest.mark.parametrize("which", LATS)
def test_equilibrium_third_moments_match_maxwell_boltzmann(which):
    """Third moments of feqH equal those of the continuous Maxwell-Boltzmann
    distribution, int f xi_a xi_b xi_c = rho (u_a u_b u_c + c_s^2 (u_a d_bc + u_b d_ac + u_c d_ab)),
    for every combination the lattice supports (D2Q9: xxy, xyy; D3Q19: the
    sums and differences of the pairs (xxy, yzz), (xzz, xyy), (yyz, xxz);
    D3Q27: each of the six a a b and x y z on its own)."""
    d, q, xi, w, opp = _lat(which)
    rng = np.random.default_rng(7)
    dl = np.eye(3)

    def mb(rho, u, a, b, c):
        return rho * (u[a] * u[b] * u[c] + CS2 * (u[a] * dl[b, c] + u[b] * dl[a, c] + u[c] * dl[a, b]))

    def m3(f, a, b, c):
        return (f * xi[:, a] * xi[:, b] * xi[:, c]).sum()

    for _ in range(10):
        rho = 0.9 + 0.2 * rng.random()
        u = 0.15 * rng.normal(size=3)
        if which == D2Q9:
            u[2] = 0
        f = oracle.feqH(which, rho, u)
        if which == D2Q9:
            for (a, b, c) in [(0, 0, 1), (0, 1, 1)]:
                assert abs(m3(f, a, b, c) - mb(rho, u, a, b, c)) < 1e-15
        elif which == D3Q27:
            for (a, b, c) in [(0, 0, 1), (0, 0, 2), (1, 1, 0), (1, 1, 2), (2, 2, 0), (2, 2, 1), (0, 1, 2)]:
                assert abs(m3(f, a, b, c) - mb(rho, u, a, b, c)) < 1e-15
        else:
            for p, qq in [((0, 0, 1), (1, 2, 2)), ((0, 2, 2), (0, 1, 1)), ((1, 1, 2), (0, 0, 2))]:
                for sgn in (1, -1):
                    got = m3(f, *p) + sgn * m3(f, *qq)
                    want = mb(rho, u, *p) + sgn * mb(rho, u, *qq)
                    assert abs(got - want) < 1e-15


def _h3_moment(which, f, idx):
    d, q, xi, w, opp = _lat(which)
    a, b, c = idx
    dl = np.eye(3)
    h = xi[:, a] * xi[:, b] * xi[:, c] - CS2 * (xi[:, a] * dl[b, c] + xi[:, b] * dl[a, c] + xi[:, c] * dl[a, b])
    return (f * h).sum()


def test_recursive_neq_third_order_special_cases_d2q9():
    """Eq. recursive2 at n = 3, evaluated by hand for simple inputs.

    u = (U, 0), Pi^neq = P (e_x e_y + e_y e_x):  a3_xxy = 2 U P, a3_xyy = 0.
    u = (U, V), Pi^neq = diag(A, B):             a3_xxy = V A, a3_xyy = U B.
    """
    U, V, P, A, B = 0.07, -0.04, 3e-3, 2e-3, -5e-3
    pn = np.zeros((3, 3)); pn[0, 1] = pn[1, 0] = P
    f = oracle.fneqH(D2Q9, [U, 0, 0], pn)
    assert abs(_h3_moment(D2Q9, f, (0, 0, 1)) - 2 * U * P) < 1e-17
    assert abs(_h3_moment(D2Q9, f, (0, 1, 1))) < 1e-17
    pn = np.diag([A, B, 0.0])
    f = oracle.fneqH(D2Q9, [U, V, 0], pn)
    assert abs(_h3_moment(D2Q9, f, (0, 0, 1)) - V * A) < 1e-17
    assert abs(_h3_moment(D2Q9, f, (0, 1, 1)) - U * B) < 1e-17
    # fneqH carries no mass and no momentum
    assert abs(f.sum()) < 1e-17
    _, _, xi, _, _ = _lat(D2Q9)
    assert np.abs((f[:, None] * xi).sum(0)).max() < 1e-17


def test_recursive_neq_third_order_special_cases_d3q19():
    """As above on D3Q19, through the supported sum/difference combinations.

    u = (U, 0, 0), Pi^neq = P (e_x e_y + e_y e_x): a3_xxy = 2UP, all other
    supported a3 components vanish, so (xxy +- yzz) moments are both 2UP.
    u = (0, V, 0), Pi^neq = diag(A, 0, C):  a3_xxy = V A, a3_yzz = V C.
    """
    U, V, P, A, Cc = 0.07, -0.04, 3e-3, 2e-3, -5e-3
    pn = np.zeros((3, 3)); pn[0, 1] = pn[1, 0] = P
    f = oracle.fneqH(D3Q19, [U, 0, 0], pn)
    s = _h3_moment(D3Q19, f, (0, 0, 1)) + _h3_moment(D3Q19, f, (1, 2, 2))
    dlt = _h3_moment(D3Q19, f, (0, 0, 1)) - _h3_moment(D3Q19, f, (1, 2, 2))
    assert abs(s - 2 * U * P) < 1e-17 and abs(dlt - 2 * U * P) < 1e-17
    for p, qq in [((0, 2, 2), (0, 1, 1)), ((1, 1, 2), (0, 0, 2))]:
        assert abs(_h3_moment(D3Q19, f, p) + _h3_moment(D3Q19, f, qq)) < 1e-17
        assert abs(_h3_moment(D3Q19, f, p) - _h3_moment(D3Q19, f, qq)) < 1e-17
    pn = np.diag([A, 0.0, Cc])
    f = oracle.fneqH(D3Q19, [0, V, 0], pn)
    s = _h3_moment(D3Q19, f, (0, 0, 1)) + _h3_moment(D3Q19, f, (1, 2, 2))
    dlt = _h3_moment(D3Q19, f, (0, 0, 1)) - _h3_moment(D3Q19, f, (1, 2, 2))
    assert abs(s - V * (A + Cc)) < 1e-17
    assert abs(dlt - V * (A - Cc)) < 1e-17


@pytest.mark.parametrize("which", LATS)
@pytest.mark.parametrize("chi", [0.1, 0.5, 1.3])
def test_sponge_homogeneous_cell_decay(which, chi):
    """In a cell, Eq. spongeLB with Eq. dampingLBM and n = m = 1/2 relaxes
    rho - rho_ref and j - rho_ref u_ref by exactly (1 - chi) / (1 + chi / 2)."""
    d, q, xi, w, opp = _lat(which)
    rho_ref = 1.0
    u_ref = np.array([0.03, -0.01, 0.02 if d == 3 else 0.0])
    for seed in range(5):
        f = _random_f(which, seed)
        r0, j0, _ = _moments(which, f)
        out = oracle.collide(which, f, 0.8, chi=chi, rho_ref=rho_ref, u_ref=u_ref)
        r1, j1, _ = _moments(which, out)
        fac = (1 - chi) / (1 + chi / 2)
        assert abs((r1 - rho_ref) - fac * (r0 - rho_ref)) < 1e-15
        assert np.abs((j1 - rho_ref * u_ref) - fac * (j0 - rho_ref * u_ref)).max() < 1e-15


def test_sponge_profile_shape():
    """sigma(x) of Sec. II.C: zero at both ends, maximum exactly 1 at 80% of the layer."""
    for W in (8, 32, 100):
        assert oracle.sigma(0, W) == 0.0
        assert oracle.sigma(W, W) == 0.0
        assert abs(oracle.sigma(0.8 * W, W) - 1.0) < 1e-14
        xs = np.linspace(0, W, 2001)
        vals = np.array([oracle.sigma(x, W) for x in xs])
        assert vals.max() <= 1.0 + 1e-14
        assert abs(xs[vals.argmax()] - 0.8 * W) <= W / 1000
        assert (vals >= 0).all()


def test_splitmix64_published_vectors(repo_root):
    path = os.path.join(repo_root, "tests", "golden", "splitmix64_seed1234567.txt")
    want = [int(l) for l in open(path) if l.strip() and not l.startswith("#")]
    G = 0x9E3779B97F4A7C15
    got = [oracle.splitmix64((1234567 + k * G) % 2 ** 64) for k in range(len(want))]
    assert got == want
    from paper_1710_02065_gb300 import inputs
    got_np = inputs.splitmix64_np(np.array([(1234567 + k * G) % 2 ** 64 for k in range(5)], dtype=np.uint64))
    assert [int(v) for v in got_np] == want
    c = 123456789
    assert oracle.u01(c) == float(inputs.u01_np(np.array([c], dtype=np.uint64))[0])


def test_circular_sponge_profile_covers_corners():
    """Radial layer (Sec. III cylinder setup): zero inside r0, the polynomial
    profile up to its maximum at r0 + 0.8 W, chi_max beyond (domain corners)."""
    P = oracle.Problem(D2Q9, (101, 101), 0.7)
    P.set_radial_sponge((50, 50), 30.0, 15.0, 0.6)
    assert P.chi(50, 50) == 0.0
    assert P.chi(50 + 30, 50) == 0.0
    assert abs(P.chi(50 + 42, 50) - 0.6) < 1e-12          # d = 12 = 0.8 W
    assert abs(P.chi(50 + 36, 50) - 0.6 * oracle.sigma(6.0, 15.0)) < 1e-15
    assert P.chi(0, 0) == 0.6 and P.chi(100, 100) == 0.6  # corners
    # radially symmetric
    assert abs(P.chi(50, 50 + 36) - P.chi(50 + 36, 50)) < 1e-15


def test_recursive_neq_third_order_special_cases_d3q27():
    """Eq. recursive2 at n = 3 on D3Q27, every supported component on its own.
    With u = (U, V, W) and Pi^neq whose only entry is P_yz = P_zy = P,
    a_abc = u_a P_bc + u_b P_ac + u_c P_ab gives a_xyz = U P, a_yyz = 2 V P,
    a_zzy = 2 W P and zero for xxy, xxz, yyx, zzx."""
    U, V, W, P = 0.07, -0.04, 0.03, 3e-3
    pn = np.zeros((3, 3)); pn[1, 2] = pn[2, 1] = P
    f = oracle.fneqH(D3Q27, [U, V, W], pn)
    want = {(0, 1, 2): U * P, (1, 1, 2): 2 * V * P, (2, 2, 1): 2 * W * P,
            (0, 0, 1): 0.0, (0, 0, 2): 0.0, (1, 1, 0): 0.0, (2, 2, 0): 0.0}
    for idx, val in want.items():
        assert abs(_h3_moment(D3Q27, f, idx) - val) < 1e-17, idx
    # the D3Q19 lattice cannot carry x y z: its H_xyz vanishes on every velocity
    _, _, xi19, _, _ = _lat(D3Q19)
    assert np.all(xi19[:, 0] * xi19[:, 1] * xi19[:, 2] == 0)
