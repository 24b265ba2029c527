"""Pins of the oracle's whole evaluation path against closed forms, convergence and its own
two summation orders (Secs. 2, 3.2, 3.3)."""
import numpy as np
import pytest

import oracle
import workloads
from sphere_exact import dl_exact, rigid, sl_exact

SPHERE = workloads.unit_sphere()


def test_plain_sums_match_closed_forms_away_from_surface():
    y = np.array([[0.1, 0.2, -0.3], [1.6, 0.4, 0.2], [0.0, 0.0, 2.5], [-0.2, 0.5, 0.1], [0.0, 0.0, 0.0]])
    b = np.linalg.norm(y, axis=1) - 1
    errs = []
    for inv in (16, 32):
        x, n, w = oracle.quadrature(SPHERE, 1 / inv)
        u, v = oracle.plain(x, n, w, rigid(x), rigid(x), y)
        errs.append((np.abs(u - sl_exact(y)).max(), np.abs(v - dl_exact(y, b)).max()))
    assert errs[1][0] < 5e-8 and errs[1][1] < 1e-7
    assert errs[0][0] > 10 * errs[1][0]


def test_single_layer_of_normal_vanishes():
    """(1/8pi) int S n dS = 0: the identity that makes the SL subtraction exact."""
    x, n, w = oracle.quadrature(workloads.Shape((0.0, 0.0, 0.0), (1.0, 0.8, 0.6)), 1 / 32)
    y = np.array([[0.1, 0.1, 0.1], [1.8, -0.3, 0.4]])
    u, _ = oracle.plain(x, n, w, n, n, y)
    assert np.abs(u).max() < 1e-6


def near_band_errors(inv, rho, count=300, seed=7):
    h = 1 / inv
    x, n, w = oracle.quadrature(SPHERE, h)
    y, _, _, _ = workloads.near_band_targets(SPHERE, count, 4 * h, np.random.default_rng(seed))
    x0, n0, b = oracle.closest_point(SPHERE, y)
    u, v, nfail = oracle.evaluate(x, n, w, rigid(x), rigid(x), y, x0, n0, b, rigid(x0), rigid(x0), h, rho)
    assert nfail == 0
    return np.abs(u - sl_exact(y)).max(), np.abs(v - dl_exact(y, b)).max()


def test_fifth_order_convergence_rho345():
    """Sec. 2.2: with delta = rho h the combined error is about O(h^5)."""
    e = [near_band_errors(inv, (3, 4, 5)) for inv in (16, 32, 64)]
    for layer in (0, 1):
        r1, r2 = e[0][layer] / e[1][layer], e[1][layer] / e[2][layer]
        assert r1 > 20 and r2 > 20, (layer, e)
    assert e[2][0] < 1e-9 and e[2][1] < 1e-6


def test_accuracy_rho234():
    e = [near_band_errors(inv, (2, 3, 4)) for inv in (16, 32, 64)]
    assert e[0][0] < 2e-5 and e[1][0] < 1e-6 and e[2][0] < 3e-8
    assert e[0][1] < 3e-4 and e[1][1] < 1e-5 and e[2][1] < 1e-6


def test_on_surface_targets():
    """Targets at the nodes (b = 0, chi = 1/2)."""
    h = 1 / 32
    x, n, w = oracle.quadrature(SPHERE, h)
    sel = np.arange(0, len(w), 37)
    y = x[sel]
    x0, n0, b = oracle.closest_point(SPHERE, y)
    assert (b == 0).all()
    u, v, nfail = oracle.evaluate(x, n, w, rigid(x), rigid(x), y, x0, n0, b, rigid(x0), rigid(x0), h, (3, 4, 5))
    assert nfail == 0
    assert np.abs(u - sl_exact(y)).max() < 3e-7
    assert np.abs(v - dl_exact(y, b)).max() < 3e-5


def test_localized_equals_direct():
    """Sec. 3.3: reusing the unregularized far part changes nothing beyond rounding."""
    wl = workloads.config("sphere16")
    x, n, w = oracle.quadrature(wl.shape, wl.h)
    f = workloads.poly_eval(wl.f_coef, x)
    q = workloads.poly_eval(wl.q_coef, x)
    y = np.concatenate([x[::7], wl.extra_targets[:400]])
    x0, n0, b = oracle.closest_point(wl.shape, y)
    f0 = workloads.poly_eval(wl.f_coef, x0)
    q0 = workloads.poly_eval(wl.q_coef, x0)
    ud, vd, _ = oracle.evaluate(x, n, w, f, q, y, x0, n0, b, f0, q0, wl.h, wl.rho, mode=oracle.DIRECT)
    ul, vl, _ = oracle.evaluate(x, n, w, f, q, y, x0, n0, b, f0, q0, wl.h, wl.rho, mode=oracle.LOCALIZED)
    assert np.abs(ud - ul).max() < 1e-13 * np.abs(ud).max()
    assert np.abs(vd - vl).max() < 1e-13 * np.abs(vd).max()


def test_one_delta_error_is_first_order_and_extrapolation_removes_it():
    """u^delta - u = O(delta) near the surface (Sec. 2); the extrapolated value is far closer."""
    h = 1 / 32
    x, n, w = oracle.quadrature(SPHERE, h)
    y, _, _, _ = workloads.near_band_targets(SPHERE, 200, 2 * h, np.random.default_rng(11))
    x0, n0, b = oracle.closest_point(SPHERE, y)
    args = (x, n, w, rigid(x), rigid(x), y, x0, n0, b, rigid(x0), rigid(x0))
    e1 = [np.abs(oracle.evaluate_one_delta(*args, r * h)[1] - dl_exact(y, b)).max() for r in (3, 6)]
    assert 1.5 < e1[1] / e1[0] < 2.5  # doubling delta roughly doubles the error
    u, v, _ = oracle.evaluate(*args, h, (3, 4, 5))
    assert np.abs(v - dl_exact(y, b)).max() < 1e-3 * e1[0]


def test_far_targets_skip_subtraction():
    """Targets farther than Rc from the surface get the plain sums."""
    wl = workloads.config("sphere32")
    x, n, w = oracle.quadrature(wl.shape, wl.h)
    f = workloads.poly_eval(wl.f_coef, x)
    q = workloads.poly_eval(wl.q_coef, x)
    y = np.array([[0.0, 0.0, 2.9], [0.05, -0.1, 0.0], [3.0, 0.0, 0.1]])
    x0, n0, b = oracle.closest_point(wl.shape, y)
    Rc = 6 * wl.rho[2] * wl.h
    assert (np.abs(b) > Rc).all()
    u, v, _ = oracle.evaluate(x, n, w, f, q, y, x0, n0, b, np.zeros_like(y), np.zeros_like(y), wl.h, wl.rho)
    up, vp = oracle.plain(x, n, w, f, q, y)
    assert np.array_equal(u, up) and np.array_equal(v, vp)
