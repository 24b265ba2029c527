"""Pins of the four-delta O(delta^7) variant the paper mentions (no formula printed): the
function I4 of the delta^5 error term, the exact weights at b = 0 and the observed order."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads
from sphere_exact import dl_exact, rigid, sl_exact

SPHERE = workloads.unit_sphere()


def test_I4_is_the_next_moment_of_erfc():
    """I0, I2 of Eqs. (I0), (I2) equal int_{|l|}^inf erfc(r) (r^2 - l^2)^k dr for k = 0, 1; I4 is k = 2
    (30-digit quadrature).  The closed forms lose relative accuracy to cancellation as lambda grows
    (I2 as printed too), so the bound is 1e-12 relative plus 1e-17 absolute."""
    mp = pytest.importorskip("mpmath")
    with mp.workdps(30):  # scoped: other modules rely on their own precision
        for lam in (0.0, 0.3, 1.0, 2.2, 4.0):
            a = mp.mpf(abs(lam))
            for k, fn in ((0, oracle.I0), (1, oracle.I2), (2, oracle.I4)):
                ref = float(mp.quad(lambda r: mp.erfc(r) * (r * r - a * a) ** k, [a, a + 2, mp.inf]))
                assert abs(fn(lam) - ref) <= 1e-12 * abs(ref) + 1e-17, (k, lam, fn(lam), ref)


def test_I4_derivative_and_limits():
    """I4' = -4 lambda I2 (as I2' = -2 lambda I0), I4(0) = 2/(5 sqrt pi), I4 even and -> 0."""
    for lam in (0.2, 0.9, 1.7, 3.0):
        e = 1e-5
        d = (oracle.I4(lam + e) - oracle.I4(lam - e)) / (2 * e)
        assert abs(d + 4 * lam * oracle.I2(lam)) < 1e-8
        assert oracle.I4(-lam) == oracle.I4(lam)
    assert abs(oracle.I4(0.0) - 2 / (5 * np.sqrt(np.pi))) < 1e-16
    assert oracle.I4(8.0) < 1e-25


@pytest.mark.parametrize("rho", [(3, 4, 5, 6), (2, 3, 4, 5)])
def test_weights_at_b0_are_the_exact_rationals(rho):
    """At b = 0 the solve is sum a_k = 1, sum a_k rho_k^(2j+1) = 0 (j = 0, 1, 2), so u equals that
    rational combination of the U_k."""
    R = [[Fraction(1)] * 4] + [[Fraction(r) ** p for r in rho] for p in (1, 3, 5)]
    rhs = [Fraction(1), Fraction(0), Fraction(0), Fraction(0)]
    n = 4  # exact Gaussian elimination on [R | rhs]
    M = [row[:] + [rhs[i]] for i, row in enumerate(R)]
    for c in range(n):
        p = next(i for i in range(c, n) if M[i][c] != 0)
        M[c], M[p] = M[p], M[c]
        for i in range(n):
            if i != c and M[i][c] != 0:
                f = M[i][c] / M[c][c]
                M[i] = [a - f * b for a, b in zip(M[i], M[c])]
    alpha = [M[i][n] / M[i][i] for i in range(n)]
    U = np.eye(4)
    got = np.array([oracle.extrapolate(rho, 0.0, 1 / 32, U[:, [k]])[0][0] for k in range(4)])
    assert np.allclose(got, [float(a) for a in alpha], rtol=1e-12, atol=1e-12), (got, alpha)


def _errors(inv, rho, count=300, seed=7):
    h = 1 / inv
    x, n, w = oracle.quadrature(SPHERE, h)
    y, _, _, _ = workloads.near_band_targets(SPHERE, count, 4 * h, np.random.default_rng(seed))
    x0, n0, b = oracle.closest_point(SPHERE, y)
    u, v, nf = oracle.evaluate(x, n, w, rigid(x), rigid(x), y, x0, n0, b, rigid(x0), rigid(x0), h, rho)
    assert nf == 0
    return np.abs(u - sl_exact(y)).max(), np.abs(v - dl_exact(y, b)).max()


def test_four_deltas_converge_faster_than_three():
    """Near-band targets on the unit sphere, rigid-body densities: with rho = (3,4,5,6) the double
    layer error falls far faster than O(h^5) (ratio > 50 from h = 1/32 to 1/64, where three deltas
    give ~32) and is > 20x smaller than the three-delta error at h = 1/64."""
    e3 = [_errors(inv, (3, 4, 5)) for inv in (32, 64)]
    e4 = [_errors(inv, (3, 4, 5, 6)) for inv in (16, 32, 64)]
    assert e4[1][1] / e4[2][1] > 50, e4
    assert e4[2][1] * 20 < e3[1][1], (e4, e3)
    assert e4[2][0] < 1e-9 and e4[2][1] < 2e-8
