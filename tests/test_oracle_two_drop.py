"""Pins of the oracle's two-drop problem (Sec. 4.3, Eq. (IE-2Surf)): the interfacial force, the
local interpolation, GMRES, and the operator on the cases where it is known exactly."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import two_drop as td


def test_jump_force_is_force_free_and_splits_normal_and_tangential():
    """[f] = 2 gamma H n - grad_S gamma: normal part 2 gamma, tangential part -grad_S gamma (the
    definition of Sec. 4.3), and a closed drop feels no net force."""
    c = np.array([2.0, 0.0, td.EPS])
    x, n, w = oracle.quadrature(workloads.unit_sphere(tuple(c)), 1 / 32)
    f = td.jump_force(x, n, c[0])
    g = td.surface_tension(x, c[0])
    assert np.allclose((f * n).sum(1), 2 * g, atol=1e-14)
    tang = f - (f * n).sum(1)[:, None] * n
    grad = np.stack([2 * (x[:, 0] - c[0]), 0 * x[:, 0], 0 * x[:, 0]], 1)
    assert np.allclose(tang, -(grad - (grad * n).sum(1)[:, None] * n), atol=1e-14)
    assert np.abs((f * w[:, None]).sum(0)).max() < 1e-6  # quadrature error of the lattice rule


@pytest.mark.parametrize("inv", [16, 32])
def test_interpolation_exact_for_tangent_polynomials(inv):
    """The local fit reproduces any polynomial of total degree <= 4 in the tangent coordinates of
    the point (the fit's own space), whatever the tangent basis."""
    h = 1 / inv
    sph = workloads.unit_sphere()
    x, n, _ = oracle.quadrature(sph, h)
    rng = np.random.default_rng(3)
    p = rng.normal(size=(40, 3))
    x0, n0, _ = oracle.closest_point(sph, p)
    W = td.interp_weights(x, x0, n0, h)
    t1, t2 = td.tangent_basis(n0)
    for i in range(len(x0)):
        idx, w = W[i]
        a = rng.normal(size=15)
        d = x[idx] - x0[i]
        xi, eta = d @ t1[i] / (3.5 * h), d @ t2[i] / (3.5 * h)
        # rotate the coordinates: the fit must not depend on the tangent basis
        ang = rng.uniform(0, 2 * np.pi)
        xr, er = np.cos(ang) * xi - np.sin(ang) * eta, np.sin(ang) * xi + np.cos(ang) * eta
        vals = td.monomials(xr, er) @ a
        assert abs(w @ vals - a[0]) < 1e-11 * np.abs(a).sum()
        assert 15 <= len(idx) <= 96


def test_interpolation_converges_at_fifth_order():
    sph = workloads.unit_sphere()
    p = np.random.default_rng(5).normal(size=(60, 3))
    errs = []
    for inv in (16, 32, 64):
        h = 1 / inv
        x, n, _ = oracle.quadrature(sph, h)
        x0, n0, _ = oracle.closest_point(sph, p)
        W = td.interp_weights(x, x0, n0, h)
        fn = lambda z: np.stack([np.sin(2 * z[:, 0]) * z[:, 1], np.exp(z[:, 2]), z[:, 0] * z[:, 1] * z[:, 2]], 1)
        got = td.interp_apply(W, fn(x))
        errs.append(np.abs(got - fn(x0)).max())
    assert errs[0] / errs[1] > 16 and errs[1] / errs[2] > 16, errs
    assert errs[2] < 1e-8, errs


def test_gmres_solves_dense_systems():
    rng = np.random.default_rng(2)
    n = 60
    A = np.eye(n) * 3 + rng.normal(size=(n, n)) / np.sqrt(n)
    b = rng.normal(size=n)
    x, it, rel = td.gmres(lambda v: A @ v, b, tol=1e-12, maxit=n)
    assert rel <= 1e-12 and it < n
    assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-10
    assert np.linalg.norm(b - A @ x) <= 1.01e-12 * np.linalg.norm(b)


@pytest.fixture(scope="module")
def drops16():
    return td.TwoDrops(1 / 16)


def test_equal_viscosities_remove_the_double_layer(drops16):
    """lambda = 1: Eq. (IE-2Surf) is 2 u = rhs, the operator is twice the identity."""
    P = td.TwoDrops(1 / 16, lam=(1.0, 1.0))
    u = np.random.default_rng(4).normal(size=3 * sum(P.N))
    assert np.array_equal(P.matvec(u), 2 * u)


def test_rigid_motions_of_one_drop(drops16):
    """For a rigid motion q of drop 1 (and 0 on drop 2), the principal-value double layer on
    drop 1 is q/2 and its value at the other drop is 0 (the identity (1/8 pi) int T q n dS = chi q),
    so A u = (2 q, 0) up to the quadrature error."""
    P = drops16
    x1 = P.nodes[0][0]
    # translation: Q = q - q(x0) = 0 in every subtracted sum, only the plain far sums carry error;
    # rotation: the other drop's nodes come within 1.5e-8 of drop 1, where the method's error at
    # h = 1/16 is ~1e-4 (the near-band double-layer bar of the sphere test at this h is 3e-4)
    for q, tol2 in ((np.tile([0.3, -0.2, 0.5], (P.N[0], 1)), 1e-6), (np.cross([0.1, 0.4, -0.3], x1 - P.centers[0]), 1e-3)):
        u = np.concatenate([q.ravel(), np.zeros(3 * P.N[1])])
        a1, a2 = P.split(P.matvec(u))
        assert np.abs(a1 - 2 * q).max() < 1e-6
        assert np.abs(a2).max() < tol2


def test_solution_at_h16(drops16):
    """GMRES reaches 1e-10 in about the 13 iterations of Table 2 at h = 1/16, and the solution
    satisfies the discrete equation."""
    P = drops16
    x, it, rel = P.solve(1e-10)
    assert rel <= 1e-10 and 10 <= it <= 15, it
    r = P.rhs() - P.matvec(x)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(P.rhs())
    # the drops move apart/together only through Marangoni stresses: velocities are O(0.1)
    assert 1e-3 < np.abs(x).max() < 1.0


def test_operator_is_affine_in_the_viscosity_ratios():
    """A(lambda) u = (lambda_b + 1) u_b - 2 sum_m (lambda_m - 1) DL_m[u_m] is affine in each
    lambda_m, with the double layer of drop m weighted by drop m's own ratio: for u = (0, q),
    A(2, 3) u - A(2, 2) u = A(2, 2) u - (0, 2 q), whatever the double-layer values are."""
    P22 = td.TwoDrops(1 / 16, lam=(2.0, 2.0))
    P23 = td.TwoDrops(1 / 16, lam=(2.0, 3.0))
    x2 = P22.nodes[1][0]
    q = np.stack([np.sin(2 * x2[:, 0]) * x2[:, 1], x2[:, 2] ** 2 - x2[:, 0], np.cos(x2[:, 1]) + x2[:, 0] * x2[:, 2]], 1)
    u = np.concatenate([np.zeros(3 * P22.N[0]), q.ravel()])
    a22, a23 = P22.matvec(u), P23.matvec(u)
    expect = a22 - np.concatenate([np.zeros(3 * P22.N[0]), 2 * q.ravel()])
    assert np.abs((a23 - a22) - expect).max() <= 1e-12 * np.abs(a22).max()
    # and the double layer of drop 2 at drop 1 is not negligible for this q
    assert np.abs(a22[:3 * P22.N[0]]).max() > 1e-3
