"""Pins of the oracle's on-surface evaluation with the modified smoothing functions s#_p of
Sec. 2.1 (one delta, no extrapolation, for targets on the surface)."""
import numpy as np
import pytest

import oracle
import workloads
from sphere_exact import rigid, sl_exact

SPHERE = workloads.unit_sphere()


def _sharp_mp(mp, t):
    c = 2 / mp.sqrt(mp.pi)
    e, g = mp.erf(t), mp.exp(-t * t)
    s1 = e + c / 3 * (5 * t - 2 * t**3) * g
    s2 = e - c / 3 * (3 * t - 14 * t**3 + 4 * t**5) * g
    s3 = e - c / 9 * (9 * t + 6 * t**3 - 4 * t**5) * g
    return [s1 / t, s2 / t**3, s3 / t**5]


def test_sigma_sharp_against_mpmath():
    """s#_p(t)/t^p from the closed forms of Sec. 2.1 at 60 digits (series and closed-form branches)."""
    mp = pytest.importorskip("mpmath")
    worst = 0.0
    with mp.workdps(60):  # scoped: other modules rely on their own precision
        for t in [1e-6, 0.01, 0.3, 0.7, 0.999, 1.0, 1.001, 1.7, 2.5, 4.0, 6.0, 7.9]:
            ref = _sharp_mp(mp, mp.mpf(t))
            got = oracle.sigma_sharp(t)
            for p in range(3):
                worst = max(worst, abs(got[p] - float(ref[p])) / abs(float(ref[p])))
    assert worst < 2e-14, worst


def test_sigma_sharp_limits():
    """At t = 0: (2/sqrt pi) (8/3, 16/3, 32/45) (the t^1, t^3, t^5 coefficients of s#_p); for
    large t, s#_p -> 1, so sigma#_p -> 1/t^p."""
    c = 2 / np.sqrt(np.pi)
    assert np.allclose(oracle.sigma_sharp(0.0), c * np.array([8 / 3, 16 / 3, 32 / 45]), rtol=1e-15, atol=0)
    t = 9.0
    assert np.allclose(oracle.sigma_sharp(t), [1 / t, 1 / t**3, 1 / t**5], rtol=1e-15, atol=0)


def test_on_surface_single_layer_fifth_order():
    """Rigid-body density on the unit sphere, targets at nodes: error against the closed form of a
    translating/rotating sphere falls ~32x per halving of h (O(delta^5), delta# = 3h)."""
    errs = []
    for inv in (16, 32, 64):
        h = 1 / inv
        x, n, w = oracle.quadrature(SPHERE, h)
        y = x[np.arange(0, len(w), max(1, len(w) // 300))]
        x0, n0, b = oracle.closest_point(SPHERE, y)
        assert (b == 0).all()
        u, _, nf = oracle.evaluate_sharp(x, n, w, rigid(x), rigid(x), y, x0, n0, b, rigid(x0), rigid(x0), h,
                                         (2, 3, 4), rho_sharp=3.0)
        assert nf == 0
        errs.append(np.abs(u - sl_exact(y)).max())
    assert errs[0] / errs[1] > 20 and errs[1] / errs[2] > 20, errs
    assert errs[2] < 2e-8


def _shared_node_values(invs, rho_sharp=3.0, seed=3):
    rng = np.random.default_rng(seed)
    fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
    xc, _, _ = oracle.quadrature(SPHERE, 1 / invs[0])
    y = xc[np.arange(0, len(xc), 7)]  # nodes of the coarsest rule are nodes of every finer one
    x0, n0, b = oracle.closest_point(SPHERE, y)
    f0, q0 = workloads.poly_eval(fc, x0), workloads.poly_eval(qc, x0)
    out = []
    for inv in invs:
        h = 1 / inv
        x, n, w = oracle.quadrature(SPHERE, h)
        f, q = workloads.poly_eval(fc, x), workloads.poly_eval(qc, x)
        us, vs, _ = oracle.evaluate_sharp(x, n, w, f, q, y, x0, n0, b, f0, q0, h, (2, 3, 4), rho_sharp=rho_sharp)
        u3, v3, _ = oracle.evaluate(x, n, w, f, q, y, x0, n0, b, f0, q0, h, (2, 3, 4))
        out.append((us, vs, u3, v3))
    return out


def test_on_surface_self_convergence_and_agreement_with_extrapolation():
    """Degree-4 densities, targets at the nodes of h = 1/16 (nodes of every finer rule): the
    successive differences v_h - v_{h/2} of the s# values fall ~32x per halving for both layers
    (a double layer written in the split form with s# would converge at first order only), and the
    s# and extrapolated values approach each other at the same rate."""
    r = _shared_node_values((16, 32, 64))
    for layer in (0, 1):
        d1 = np.abs(r[0][layer] - r[1][layer]).max()
        d2 = np.abs(r[1][layer] - r[2][layer]).max()
        assert d1 / d2 > 20, (layer, d1, d2)
        g = [np.abs(r[k][layer] - r[k][layer + 2]).max() for k in range(3)]
        assert g[0] / g[1] > 15 and g[1] / g[2] > 15, (layer, g)


def test_off_surface_targets_use_the_extrapolated_method():
    h = 1 / 16
    x, n, w = oracle.quadrature(SPHERE, h)
    y, _, _, _ = workloads.near_band_targets(SPHERE, 40, 4 * h, np.random.default_rng(1))
    y = np.concatenate([y, x[:10]])
    x0, n0, b = oracle.closest_point(SPHERE, y)
    us, vs, _ = oracle.evaluate_sharp(x, n, w, rigid(x), rigid(x), y, x0, n0, b, rigid(x0), rigid(x0), h, (2, 3, 4))
    u3, v3, _ = oracle.evaluate(x, n, w, rigid(x), rigid(x), y, x0, n0, b, rigid(x0), rigid(x0), h, (2, 3, 4))
    off = b != 0
    assert off.sum() == 40
    assert np.array_equal(us[off], u3[off]) and np.array_equal(vs[off], v3[off])
    assert not np.array_equal(us[~off], u3[~off])
