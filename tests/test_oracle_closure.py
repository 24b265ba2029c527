"""Pins of the oracle of the learned closure: the reduced one- and two-delta sums (Eq. (extrap_eqn)
with fewer deltas) and the features (principal frame and curvatures of the ellipsoid, density
jets from the local least-squares fit), against exact values, identities, closed forms of
differential geometry and observed orders of convergence."""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import closure
from sphere_exact import dl_exact, rigid, sl_exact

SPHERE = workloads.unit_sphere()
ELL = workloads.Shape((0.0, 0.0, 0.0), (1.0, 0.8, 0.6))


@pytest.mark.parametrize("rho", [(2.0, 3.0, 4.0), (3.0, 4.0, 5.0)])
def test_two_delta_weights_exact_at_zero(rho):
    """At b = 0, I0 = 1/sqrt(pi) for both deltas: beta = (rho_1, -rho_0) / (rho_1 - rho_0) and
    gamma = -rho_0 rho_1 (rho_0 + rho_1) I2(0) with I2(0) = 1 / (3 sqrt(pi))."""
    beta, g, rc = oracle.reduced_weights(2, rho, 0.0, 1 / 32)
    r0, r1 = rho[0], rho[1]
    assert rc == 0
    assert beta[0] == pytest.approx(r1 / (r1 - r0), rel=1e-15)
    assert beta[1] == pytest.approx(-r0 / (r1 - r0), rel=1e-15)
    assert g == pytest.approx(-r0 * r1 * (r0 + r1) / (3 * math.sqrt(math.pi)), rel=1e-14)
    beta1, g1, _ = oracle.reduced_weights(1, rho, 0.3, 1 / 32)
    assert tuple(beta1) == (1.0, 0.0) and g1 == 0.0


def test_two_delta_weights_identities():
    """sum beta = 1 and sum beta rho I0(lambda) = 0 at every b (the c1 term cancels), and gamma is
    the same combination of rho^3 I2."""
    rho, h = (2.0, 3.0, 4.0), 1 / 64
    for b in np.linspace(-18 * h, 18 * h, 37):
        beta, g, rc = oracle.reduced_weights(2, rho, b, h)
        assert rc == 0
        i0 = [rho[k] * oracle.I0(b / (rho[k] * h)) for k in range(2)]
        i2 = [rho[k] ** 3 * oracle.I2(b / (rho[k] * h)) for k in range(2)]
        assert beta.sum() == pytest.approx(1.0, abs=1e-12 * np.abs(beta).sum())
        assert abs(beta @ i0) <= 1e-14 * np.abs(beta).sum()
        assert g == pytest.approx(beta @ i2, rel=1e-13, abs=1e-300)


def _band(shape, h, count, bmax, seed):
    y, _, _, _ = workloads.near_band_targets(shape, count, bmax, np.random.default_rng(seed))
    return y


def test_two_delta_value_with_three_delta_c2_is_the_three_delta_value():
    """From the three equations of Eq. (extrap_eqn) (u, c1, c2 solved from the one-delta sums),
    u2 - gamma c2 = u exactly: the two-delta combination and gamma are the elimination of c1 from
    the first two equations.  The one-delta reduced sum is the delta_0 sum itself."""
    h, rho = 1 / 16, (2.0, 3.0, 4.0)
    x, n, w = oracle.quadrature(ELL, h)
    rng = np.random.default_rng(3)
    fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
    f, q = workloads.poly_eval(fc, x), workloads.poly_eval(qc, x)
    y = np.concatenate([_band(ELL, h, 150, 4 * h, 11), x[::97]])
    x0, n0, b = oracle.closest_point(ELL, y)
    f0, q0 = workloads.poly_eval(fc, x0), workloads.poly_eval(qc, x0)
    U = [oracle.evaluate_one_delta(x, n, w, f, q, y, x0, n0, b, f0, q0, r * h) for r in rho]
    u3, v3, _ = oracle.evaluate(x, n, w, f, q, y, x0, n0, b, f0, q0, h, rho, mode=oracle.DIRECT)
    u2, v2, g = oracle.evaluate_reduced(2, x, n, w, f, q, y, x0, n0, b, f0, q0, h, rho)
    u1, v1, g1 = oracle.evaluate_reduced(1, x, n, w, f, q, y, x0, n0, b, f0, q0, h, rho)
    assert np.array_equal(g1, np.zeros_like(g1))
    assert np.abs(u1 - U[0][0]).max() <= 1e-13 * np.abs(U[0][0]).max()
    assert np.abs(v1 - U[0][1]).max() <= 1e-13 * np.abs(U[0][1]).max()
    for m in range(len(b)):
        A = np.array([[1.0, r * oracle.I0(b[m] / (r * h)), r**3 * oracle.I2(b[m] / (r * h))] for r in rho])
        for layer, (red, ref) in enumerate(((u2, u3), (v2, v3))):
            sol = np.linalg.solve(A, np.stack([U[k][layer][m] for k in range(3)]))
            np.testing.assert_allclose(red[m] - g[m] * sol[2], ref[m], rtol=0, atol=1e-12 * np.abs(ref).max())


def test_reduced_sums_converge_at_their_orders():
    """Against the sphere closed forms: the two-delta value is O(delta^3) (the gamma c2 term), the
    one-delta sum O(delta) (Eq. (extrap_eqn)); errors at targets |b| <= 2h for h = 1/16, 1/32, 1/64."""
    e = {1: [], 2: []}
    for inv in (16, 32, 64):
        h = 1 / inv
        x, n, w = oracle.quadrature(SPHERE, h)
        y = _band(SPHERE, h, 120, 2 * h, 5)
        x0, n0, b = oracle.closest_point(SPHERE, y)
        for K in (1, 2):
            u, v, _ = oracle.evaluate_reduced(K, x, n, w, rigid(x), rigid(x), y, x0, n0, b, rigid(x0), rigid(x0),
                                              h, (2.0, 3.0, 4.0))
            e[K].append((np.abs(u - sl_exact(y)).max(), np.abs(v - dl_exact(y, b)).max()))
    for layer in (0, 1):
        r2 = [e[2][i][layer] / e[2][i + 1][layer] for i in range(2)]
        r1 = [e[1][i][layer] / e[1][i + 1][layer] for i in range(2)]
        assert all(5.0 < r < 12.0 for r in r2), (layer, e[2])
        assert all(1.6 < r < 2.6 for r in r1), (layer, e[1])


def test_targets_beyond_the_reduced_radius_take_the_plain_sums():
    h, rho = 1 / 32, (2.0, 3.0, 4.0)
    x, n, w = oracle.quadrature(SPHERE, h)
    rng = np.random.default_rng(8)
    fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
    f, q = workloads.poly_eval(fc, x), workloads.poly_eval(qc, x)
    y = np.array([[0.0, 0.0, 0.1], [0.0, 1.7, 0.0], [0.2, 0.1, 0.3]])
    x0, n0, b = oracle.closest_point(SPHERE, y)
    for K in (1, 2):
        assert (np.abs(b) > 6 * rho[K - 1] * h).all()
        u, v, g = oracle.evaluate_reduced(K, x, n, w, f, q, y, x0, n0, b, workloads.poly_eval(fc, x0),
                                          workloads.poly_eval(qc, x0), h, rho)
        up, vp = oracle.plain(x, n, w, f, q, y)
        assert np.array_equal(u, up) and np.array_equal(v, vp) and (g == 0).all()


def test_sphere_frame_and_curvatures():
    rng = np.random.default_rng(1)
    for R in (1.0, 0.7):
        shape = workloads.Shape((0.1, -0.2, 0.3), (R, R, R))
        x0, n0 = workloads.surface_points(shape, 50, rng)
        for m in range(50):
            fr, k1, k2 = closure.principal_frame(shape, x0[m], n0[m])
            assert k1 == pytest.approx(1 / R, rel=1e-13) and k2 == pytest.approx(1 / R, rel=1e-13)
            assert np.abs(fr @ fr.T - np.eye(3)).max() < 1e-14
            assert np.allclose(np.cross(fr[0], fr[1]), fr[2], atol=1e-14)
            assert np.array_equal(fr, closure.fallback_frame(n0[m]))


def test_ellipsoid_axis_points():
    """At (a, 0, 0) of the ellipsoid (a, b, c) the normal curvatures along e_y and e_z are a/b^2 and
    a/c^2; with (1, 0.8, 0.6) the larger is along e_z."""
    fr, k1, k2 = closure.principal_frame(ELL, np.array([1.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0]))
    assert k1 == pytest.approx(1 / 0.36, rel=1e-14) and k2 == pytest.approx(1 / 0.64, rel=1e-14)
    assert abs(abs(fr[0][2]) - 1.0) < 1e-14 and abs(abs(fr[1][1]) - 1.0) < 1e-14


def _normal_curvature(shape, x0, n0, t, s=2e-4):
    """Curvature of the normal section along unit tangent t: the height z(s) of the surface over
    x0 + s t (F(x0 + s t + z n0) = 1, solved by Newton), kappa = -z''(0) by central differences."""
    c, a = np.asarray(shape.center), np.asarray(shape.axes)

    def z(sv):
        zz = 0.0
        for _ in range(60):
            p = x0 + sv * t + zz * n0 - c
            F = ((p / a) ** 2).sum() - 1
            dF = (2 * p / a**2) @ n0
            zz -= F / dF
        return zz
    return -(z(s) - 2 * z(0.0) + z(-s)) / s**2


def test_ellipsoid_principal_directions_and_curvatures():
    """At random points: the normal curvature along t1 (t2) is k1 (k2), no tangent direction
    curves more than k1 or less than k2, and k1 k2 equals the Gauss curvature of the ellipsoid,
    1 / (a^2 b^2 c^2 |p / a^2|^4)."""
    rng = np.random.default_rng(4)
    x0, n0 = workloads.surface_points(ELL, 40, rng)
    a2 = np.asarray(ELL.axes) ** 2
    for m in range(40):
        fr, k1, k2 = closure.principal_frame(ELL, x0[m], n0[m])
        assert k1 >= k2 > 0
        assert np.abs(fr @ fr.T - np.eye(3)).max() < 1e-14
        assert np.allclose(np.cross(fr[0], fr[1]), fr[2], atol=1e-14)  # (t1, t2, n0) right-handed
        assert _normal_curvature(ELL, x0[m], n0[m], fr[0]) == pytest.approx(k1, rel=2e-6)
        assert _normal_curvature(ELL, x0[m], n0[m], fr[1]) == pytest.approx(k2, rel=2e-6)
        for th in np.linspace(0.1, 3.0, 7):
            t = math.cos(th) * fr[0] + math.sin(th) * fr[1]
            kn = _normal_curvature(ELL, x0[m], n0[m], t)
            assert k2 * (1 - 2e-6) <= kn <= k1 * (1 + 2e-6)
        g = x0[m] / a2
        assert k1 * k2 == pytest.approx(1.0 / (a2.prod() * (g @ g) ** 2), rel=1e-12)


def test_jets_exact_for_a_polynomial_in_the_tangent_coordinates():
    """Node values that are a polynomial of degree <= 4 in (xi, eta) of x0 are fitted exactly: the
    jets are that polynomial's derivatives i! j! c_ij."""
    h = 1 / 32
    x, n, w = oracle.quadrature(ELL, h)
    rng = np.random.default_rng(6)
    x0, n0 = workloads.surface_points(ELL, 5, rng)
    for m in range(5):
        fr, _, _ = closure.principal_frame(ELL, x0[m], n0[m])
        C = rng.standard_normal((15, 3))
        d = x - x0[m]
        xi, eta = d @ fr[0] / h, d @ fr[1] / h
        vals_local = sum(np.outer(xi**i * eta**j, C[k]) for k, (i, j) in enumerate(closure.MONOMIALS))
        vals = vals_local @ fr  # back to x, y, z components
        J = closure.density_jets(x, vals, x0[m], fr, h)
        assert J is not None
        fact = np.array([math.factorial(i) * math.factorial(j) for (i, j) in closure.MONOMIALS])
        np.testing.assert_allclose(J, C * fact[:, None], rtol=0, atol=1e-9 * np.abs(C).max() * 24)


def test_jets_match_surface_derivatives_on_the_sphere():
    """For a smooth density on the unit sphere: the fitted value, first and second tangent-plane
    derivatives approach f(x0), h (grad f . t_a) and h^2 (t_a^T H t_b - delta_ab (grad f . n0) / R)
    (the Monge patch z(xi, eta) of a sphere of radius R has z_ab = -delta_ab / R)."""
    rng = np.random.default_rng(12)
    coef = workloads.density_coeffs(rng)
    errs = []
    for inv in (32, 64):
        h = 1 / inv
        x, n, w = oracle.quadrature(SPHERE, h)
        vals = workloads.poly_eval(coef, x)
        x0, n0 = workloads.surface_points(SPHERE, 6, np.random.default_rng(2))
        e = [0.0, 0.0, 0.0]
        for m in range(6):
            fr, _, _ = closure.principal_frame(SPHERE, x0[m], n0[m])
            J = closure.density_jets(x, vals, x0[m], fr, h)
            f0 = workloads.poly_eval(coef, x0[m][None])[0]
            G = workloads.poly_jacobian(coef, x0[m][None])[0]
            eps = 1e-4
            H = np.stack([(workloads.poly_jacobian(coef, (x0[m] + eps * np.eye(3)[k])[None])[0]
                           - workloads.poly_jacobian(coef, (x0[m] - eps * np.eye(3)[k])[None])[0]) / (2 * eps)
                          for k in range(3)], axis=-1)  # H[i, j, k] = d2 f_i / dx_j dx_k
            fn = G @ n0[m]
            ref0 = fr @ f0
            ref1 = [fr @ (G @ fr[a]) * h for a in range(2)]
            ref2 = {}
            for a in range(2):
                for bb in range(2):
                    ref2[(a, bb)] = fr @ (np.einsum("ijk,j,k->i", H, fr[a], fr[bb]) - (a == bb) * fn) * h * h
            e[0] = max(e[0], np.abs(J[0] - ref0).max() / np.abs(ref0).max())
            e[1] = max(e[1], max(np.abs(J[1 + a] - ref1[a]).max() for a in range(2)) * inv)
            j2 = {(0, 0): J[3], (0, 1): J[4], (1, 0): J[4], (1, 1): J[5]}
            e[2] = max(e[2], max(np.abs(j2[k] - ref2[k]).max() for k in ref2) * inv * inv)
        errs.append(e)
    assert errs[1][0] < 1e-8 and errs[1][1] < 1e-5 and errs[1][2] < 1e-3, errs
    assert errs[0][1] > 3 * errs[1][1] and errs[0][2] > 3 * errs[1][2], errs


def test_features_scale_and_validity():
    h, rho = 1 / 16, (2.0, 3.0, 4.0)
    x, n, w = oracle.quadrature(ELL, h)
    rng = np.random.default_rng(13)
    fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
    f, q = workloads.poly_eval(fc, x), workloads.poly_eval(qc, x)
    y = np.concatenate([_band(ELL, h, 60, 20 * h, 3), [[0.0, 0.0, 0.0]]])
    x0, n0, b = oracle.closest_point(ELL, y)
    for nd in (1, 2):
        geom, frames, jets, scale = closure.features(ELL, x, f, q, x0, n0, b, h, rho, nd)
        Rc = 6 * rho[nd - 1] * h
        near = np.abs(b) <= Rc
        assert ((scale > 0).all(axis=1) == near).all()
        for layer in range(2):
            ok = scale[:, layer] > 0
            assert np.allclose(np.abs(jets[layer][ok]).max(axis=1), 1.0)
            assert (jets[layer][~ok] == 0).all()
        assert np.allclose(geom[:, 0], b / (rho[0] * h)) and (geom[:, 3] == rho[0]).all() and (geom[:, 4] == rho[1]).all()


def test_targets_and_apply_are_inverse():
    """Applying the training targets themselves as the network's output gives back the three-delta
    values (ndelta = 1 and 2) wherever a target has weight; elsewhere the reduced value is kept."""
    h, rho = 1 / 16, (2.0, 3.0, 4.0)
    x, n, w = oracle.quadrature(SPHERE, h)
    rng = np.random.default_rng(14)
    fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
    f, q = workloads.poly_eval(fc, x), workloads.poly_eval(qc, x)
    y = _band(SPHERE, h, 80, 10 * h, 9)
    x0, n0, b = oracle.closest_point(SPHERE, y)
    f0, q0 = workloads.poly_eval(fc, x0), workloads.poly_eval(qc, x0)
    u3, v3, _ = oracle.evaluate(x, n, w, f, q, y, x0, n0, b, f0, q0, h, rho)
    for nd in (1, 2):
        ur, vr, g = oracle.evaluate_reduced(nd, x, n, w, f, q, y, x0, n0, b, f0, q0, h, rho)
        geom, frames, jets, scale = closure.features(SPHERE, x, f, q, x0, n0, b, h, rho, nd)
        (cs, cd), (ws, wd) = closure.targets(frames, scale, h, nd, ur, vr, g, u3, v3, rho)
        ua, va = closure.apply(frames, scale, h, nd, ur, vr, g, cs, cd)
        for got, red, ref, wt in ((ua, ur, u3, ws), (va, vr, v3, wd)):
            on = wt > 0
            assert on.sum() > 20
            np.testing.assert_allclose(got[on], ref[on], rtol=0, atol=1e-12 * np.abs(ref).max())
            np.testing.assert_array_equal(got[~on & (scale[:, 0] == 0)], red[~on & (scale[:, 0] == 0)])
