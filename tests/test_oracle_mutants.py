"""Planted mistakes in the oracle, on the CPU: each test compiles a copy of the oracle's C source
with one plausible slip (a dropped term, a wrong sign or coefficient, transposed operands) and
checks that the pins of the oracle's tests catch it, while the unedited copy passes them all.
The pins used here are those of test_oracle_method.py (the sphere closed forms for rigid-body
densities at near-band targets and at the nodes; the equality of the localized and direct forms,
Sec. 3.3), of test_oracle_functions.py (I0(0) = 1/sqrt(pi), I2(0) = 1/(3 sqrt(pi)),
I0' = -erfc, I2' = -2 lambda I0) and of test_oracle_quadrature.py (Table 1's node count, the
area).  A constant factor in I0 or I2 leaves the extrapolated value
unchanged (it rescales a column of the system of Eq. (extrap_eqn), so only c1 or c2 changes): only
the function-level pins see it."""
import math
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads
from sphere_exact import dl_exact, rigid, sl_exact

SRC = os.path.join(os.path.dirname(oracle.__file__), "ers_oracle.c")
TREE_SRC = os.path.join(os.path.dirname(oracle.__file__), "ers_treecode.c")
SPHERE = workloads.unit_sphere()

# (what the slip is, text in ers_oracle.c, replacement); the first occurrence is edited, which
# is the one ora_eval (three deltas) runs.
MUTANTS = [
    ("single layer: the d (d.g) s2/r^3 term dropped",
     "acc[i] += (k1 * g[i] + k3 * dg * d[i]) * w;", "acc[i] += (k1 * g[i]) * w;"),
    ("double layer: sign of the stresslet",
     "double T = -6.0 * (t1 * k3 + (t2 - r2mb2 * t1) * k5);", "double T = 6.0 * (t1 * k3 + (t2 - r2mb2 * t1) * k5);"),
    ("double layer: (r^2 - b^2) written as (r^2 + b^2)",
     "double r2mb2 = r * r - b * b;", "double r2mb2 = r * r + b * b;"),
    ("double layer: n0 and n(x) transposed",
     "ora_dl_term(r, delta, tc, bm, nm0, xh, Q, nj, w[j], snear_v[k], 0);",
     "ora_dl_term(r, delta, tc, bm, nj, xh, Q, nm0, w[j], snear_v[k], 0);"),
    ("double layer: one index of t2 wrong (xh_i xh_j n_k -> xh_i xh_j n_j)",
     "double t2 = b * (xi[i] * xi[j] * ni[k] +", "double t2 = b * (xi[i] * xi[j] * ni[j] +"),
    ("I2: coefficient 2/3 -> 1/3",
     "return 2.0 / 3.0 * ((0.5 - l * l)", "return 1.0 / 3.0 * ((0.5 - l * l)"),
    ("I2: sign of lambda^2 in (1/2 - lambda^2)",
     "return 2.0 / 3.0 * ((0.5 - l * l)", "return 2.0 / 3.0 * ((0.5 + l * l)"),
    ("I0: sign of the erfc term",
     "return exp(-l * l) / ORA_SQRTPI - l * erfc(l);", "return exp(-l * l) / ORA_SQRTPI + l * erfc(l);"),
    ("chi: inside and outside swapped",
     "double chi = (bm < 0.0) ? 1.0 : ((bm > 0.0) ? 0.0 : 0.5);",
     "double chi = (bm < 0.0) ? 0.0 : ((bm > 0.0) ? 1.0 : 0.5);"),
    ("single-layer subtraction: sign of (f(x0).n0) n",
     "g[i] = f[3 * j + i] - fn0 * nj[i];", "g[i] = f[3 * j + i] + fn0 * nj[i];"),
    ("double-layer subtraction: q(x0) not subtracted",
     "Q[i] = q[3 * j + i] - qm0[i];", "Q[i] = q[3 * j + i];"),
    ("s2/t^3 series (t < 1/2): sign of its terms",
     "if (nn >= 1) s2 += -sgn * (2.0 * nn)", "if (nn >= 1) s2 += sgn * (2.0 * nn)"),
    ("quadrature: the 1/|n_k| factor of the weight dropped",
     "w[count] = psi / fabs(nn[k]) * h * h;", "w[count] = psi * h * h;"),
    ("quadrature: partition of unity taken along the wrong axis",
     "double psi = beta[k] / sb;", "double psi = beta[(k + 1) % 3] / sb;"),
    ("s3: coefficient of t^3 in the closed form 2/3 -> 1/3",
     "double s3 = e - c * (t + 2.0 / 3.0 * t * t * t) * g;", "double s3 = e - c * (t + 1.0 / 3.0 * t * t * t) * g;"),
]


def _compile(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    lib = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(lib), str(src), TREE_SRC,
                    "-lm"], check=True)
    return oracle.bind(ctypes.CDLL(str(lib)))


def _pins():
    """(name, passed) for each pin, with the library currently loaded in the oracle package."""
    out = []
    # near-band targets |b| <= 4h (the bounds of test_accuracy_rho234), then nodes (b = 0, the
    # bounds of test_on_surface_targets)
    for inv, rho, nodes, sl_tol, dl_tol in ((16, (2, 3, 4), False, 2e-5, 3e-4), (32, (2, 3, 4), False, 1e-6, 1e-5),
                                            (32, (3, 4, 5), True, 3e-7, 3e-5)):
        h = 1 / inv
        x, n, w = oracle.quadrature(SPHERE, h)
        if nodes:
            y = x[np.arange(0, len(w), 37)]
        else:
            y, _, _, _ = workloads.near_band_targets(SPHERE, 300, 4 * h, np.random.default_rng(7))
        x0, n0, b = oracle.closest_point(SPHERE, y)
        u, v, nfail = oracle.evaluate(x, n, w, rigid(x), rigid(x), y, x0, n0, b, rigid(x0), rigid(x0), h, rho)
        where = f"h = 1/{inv}, {'nodes' if nodes else 'band'}"
        out.append((f"sphere closed form, single layer, {where}", nfail == 0 and np.abs(u - sl_exact(y)).max() < sl_tol))
        out.append((f"sphere closed form, double layer, {where}",
                    nfail == 0 and np.abs(v - dl_exact(y, b)).max() < dl_tol))
    wl = workloads.config("sphere16")
    x, n, w = oracle.quadrature(wl.shape, wl.h)
    f, q = workloads.poly_eval(wl.f_coef, x), workloads.poly_eval(wl.q_coef, x)
    y = np.concatenate([x[::7], wl.extra_targets[:300]])
    x0, n0, b = oracle.closest_point(wl.shape, y)
    f0, q0 = workloads.poly_eval(wl.f_coef, x0), workloads.poly_eval(wl.q_coef, x0)
    ud, vd, _ = oracle.evaluate(x, n, w, f, q, y, x0, n0, b, f0, q0, wl.h, wl.rho, mode=oracle.DIRECT)
    ul, vl, _ = oracle.evaluate(x, n, w, f, q, y, x0, n0, b, f0, q0, wl.h, wl.rho, mode=oracle.LOCALIZED)
    out.append(("localized = direct", np.abs(ud - ul).max() < 1e-13 * np.abs(ud).max()
                and np.abs(vd - vl).max() < 1e-13 * np.abs(vd).max()))
    # quadrature (Sec. 2.2): Table 1's node count for the spheroid (1, 1/2, 1/2) at h = 1/32, and
    # the weights integrate the unit sphere's area
    _, _, w = oracle.quadrature(workloads.Shape((0.0, 0.0, 0.0), (1.0, 0.5, 0.5)), 1 / 32)
    out.append(("Table 1 node count", len(w) == 6958))
    _, _, w = oracle.quadrature(SPHERE, 1 / 64)
    out.append(("weights integrate the area", abs(w.sum() - 4 * np.pi) < 5e-9))
    sp = math.sqrt(math.pi)
    ok = abs(oracle.I0(0.0) - 1 / sp) < 1e-16 and abs(oracle.I2(0.0) - 1 / (3 * sp)) < 1e-16
    for lam in (0.3, 1.1, 2.5):
        eps = 1e-6
        d0 = (oracle.I0(lam + eps) - oracle.I0(lam - eps)) / (2 * eps)
        d2 = (oracle.I2(lam + eps) - oracle.I2(lam - eps)) / (2 * eps)
        ok = ok and abs(d0 + math.erfc(lam)) < 1e-9 and abs(d2 + 2 * lam * oracle.I0(lam)) < 1e-9
    out.append(("I0, I2 values at 0 and derivative identities", ok))
    return out


def _with_library(lib):
    saved = oracle._lib
    oracle._lib = lib
    try:
        return _pins()
    finally:
        oracle._lib = saved


def test_unedited_copy_passes_every_pin(tmp_path):
    lib = _compile(tmp_path, "unedited", open(SRC).read())
    failed = [name for name, ok in _with_library(lib) if not ok]
    assert not failed, failed


@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, what, old, new):
    text = open(SRC).read()
    assert old in text, f"the text to edit is not in the oracle: {old}"
    lib = _compile(tmp_path, "mutant", text.replace(old, new, 1))
    results = _with_library(lib)
    caught = [name for name, ok in results if not ok]
    print(what, "->", caught)
    assert caught, f"no pin catches: {what}"


# Slips in the treecode (ers_treecode.c, Sec. 3.4), against the pins of test_oracle_treecode.py.
TREE_SRC_TEXT_MUTANTS = [
    ("barycentric weights: end points not halved",
     "double wk = ((k & 1) ? -1.0 : 1.0) * ((k == 0 || k == p) ? 0.5 : 1.0);",
     "double wk = ((k & 1) ? -1.0 : 1.0) * 1.0;"),
    ("barycentric weights: alternating sign dropped",
     "double wk = ((k & 1) ? -1.0 : 1.0) * ((k == 0 || k == p) ? 0.5 : 1.0);",
     "double wk = 1.0 * ((k == 0 || k == p) ? 0.5 : 1.0);"),
    ("modified weights: density q_a n_b transposed to q_b n_a",
     "g[6 + 3 * a + b] = q[3 * j + a] * nrm[3 * j + b] * w[j];",
     "g[6 + 3 * a + b] = q[3 * j + b] * nrm[3 * j + a] * w[j];"),
    # (q0 subtracted with transposed indices, q0_b Wn_a, is no slip: the contraction with d_a d_b
    # is symmetric in a, b)
    ("cluster sum: q0 times the f weights instead of the n weights",
     "t->q0[a] * Wk[3 + b]", "t->q0[a] * Wk[b]"),
    ("cluster sum: sign of the single-layer subtraction",
     "g[i] = Wk[i] - t->fn0 * Wk[3 + i];", "g[i] = Wk[i] + t->fn0 * Wk[3 + i];"),
    ("MAC without the near-radius condition",
     "if (C->rc <= X->theta * R && R - C->rc > X->Racc) {", "if (C->rc <= X->theta * R) {"),
    ("Lagrange basis at Chebyshev points of the first kind",
     "for (int k = 0; k <= p; ++k) s[k] = c + hw * cos(k * ORA_TC_PI / p);",
     "for (int k = 0; k <= p; ++k) s[k] = c + hw * cos((2 * k + 1) * ORA_TC_PI / (2 * p + 2));"),
]


def _compile_tree(tmp_path, name, tree_text):
    src = tmp_path / f"{name}_tree.c"
    src.write_text(tree_text)
    lib = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(lib), SRC, str(src), "-lm"],
                   check=True)
    return oracle.bind(ctypes.CDLL(str(lib)))


def _tree_pins(stop_at_failure=False):
    import test_oracle_treecode as T
    ell = oracle.quadrature(T.ELL, 1 / 32)
    checks = [("Lagrange basis p = 2", lambda: T.test_lagrange_basis(2)),
              ("Lagrange basis p = 5", lambda: T.test_lagrange_basis(5)),
              ("modified-weight moments p = 3", lambda: T.test_modified_weights_moments(ell, 3)),
              ("theta -> 0 is the direct evaluation", T.test_theta_zero_is_the_direct_evaluation),
              ("every node counted once", lambda: T.test_every_node_counted_once((2.0, 3.0, 4.0))),
              ("spectral decay with p", T.test_error_decays_spectrally_with_degree)]
    out = []
    for name, fn in checks:
        try:
            fn()
            out.append((name, True))
        except AssertionError:
            out.append((name, False))
            if stop_at_failure:
                break
    return out


def _with_library_tree(lib, stop_at_failure=False):
    saved = oracle._lib
    oracle._lib = lib
    try:
        return _tree_pins(stop_at_failure)
    finally:
        oracle._lib = saved


def test_unedited_treecode_copy_passes_every_pin(tmp_path):
    lib = _compile_tree(tmp_path, "unedited", open(TREE_SRC).read())
    failed = [name for name, ok in _with_library_tree(lib) if not ok]
    assert not failed, failed


@pytest.mark.parametrize("what,old,new", TREE_SRC_TEXT_MUTANTS, ids=[m[0] for m in TREE_SRC_TEXT_MUTANTS])
def test_planted_treecode_mistake_fails_a_pin(tmp_path, what, old, new):
    text = open(TREE_SRC).read()
    assert old in text, f"the text to edit is not in the treecode oracle: {old}"
    lib = _compile_tree(tmp_path, "mutant", text.replace(old, new, 1))
    caught = [name for name, ok in _with_library_tree(lib, True) if not ok]
    print(what, "->", caught)
    assert caught, f"no pin catches: {what}"


# Slips in the two-drop oracle (oracle/two_drop.py, Sec. 4.3), against the pins of
# test_oracle_two_drop.py (a Python module: the edited source is executed as a module of its own).
TWO_DROP_MUTANTS = [
    ("jump force: sign of the surface gradient", "return 2.0 * g[:, None] * H * n - grad_s",
     "return 2.0 * g[:, None] * H * n + grad_s"),
    ("jump force: surface gradient not projected on the tangent plane",
     "grad_s = grad - (grad * n).sum(1)[:, None] * n", "grad_s = grad"),
    ("local fit: degree 3 instead of 4", "cols = [xi ** (d - b) * eta ** b for d in range(deg + 1) for b in range(d + 1)]",
     "cols = [xi ** (d - b) * eta ** b for d in range(deg) for b in range(d + 1)]"),
    # (a first tangent not orthogonalized against n0 is no slip: the fit is then a polynomial in
    # another local chart of the surface, just as accurate)
    ("local fit: the second tangent equal to the first",
     "t2 = np.cross(n0, t1)", "t2 = t1.copy()"),
    ("GMRES: sign of the rotated residual", "g[k + 1] = -sn[k] * g[k]", "g[k + 1] = sn[k] * g[k]"),
    ("GMRES: previous rotation applied with the wrong sign",
     "H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]", "H[i + 1, k] = sn[i] * H[i, k] + cs[i] * H[i + 1, k]"),
    ("operator: (lambda_b - 1) u_b instead of (lambda_b + 1) u_b",
     "out.append((self.lam[b] + 1.0) * us[b] - v)", "out.append((self.lam[b] - 1.0) * us[b] - v)"),
    ("operator: double layer of the other drop with its own viscosity",
     "v = sum(2.0 * (self.lam[m] - 1.0) * self.layer(m, b, None, us[m], 1) for m in range(2))",
     "v = sum(2.0 * (self.lam[b] - 1.0) * self.layer(m, b, None, us[m], 1) for m in range(2))"),
]


def _two_drop_pins(mod, stop_at_failure=False):
    """(name, passed) per pin, cheapest first; with stop_at_failure the list ends at the first
    failing pin (enough to show that a slip is caught)."""
    import test_oracle_two_drop as T
    saved = T.td
    T.td = mod
    try:
        checks = [("jump force", T.test_jump_force_is_force_free_and_splits_normal_and_tangential),
                  ("GMRES on dense systems", T.test_gmres_solves_dense_systems),
                  ("fit exact on its polynomials", lambda: T.test_interpolation_exact_for_tangent_polynomials(16)),
                  ("fit converges at fifth order", T.test_interpolation_converges_at_fifth_order),
                  ("lambda = 1 gives 2 I", lambda: T.test_equal_viscosities_remove_the_double_layer(None)),
                  # the operator at h = 1/16 with unequal viscosities: rigid motions of one drop,
                  # and the affine dependence on the ratios
                  ("rigid motions", lambda: T.test_rigid_motions_of_one_drop(mod.TwoDrops(1 / 16, lam=(2.0, 3.0)))),
                  ("affine in the viscosity ratios", T.test_operator_is_affine_in_the_viscosity_ratios)]
        out = []
        for name, fn in checks:
            try:
                fn()
                out.append((name, True))
            except (AssertionError, ValueError, np.linalg.LinAlgError):
                out.append((name, False))
                if stop_at_failure:
                    break
        return out
    finally:
        T.td = saved


def _two_drop_module(text):
    import types
    from oracle import two_drop
    mod = types.ModuleType("two_drop_copy")
    mod.__file__ = two_drop.__file__
    exec(compile(text, two_drop.__file__, "exec"), mod.__dict__)
    return mod


def test_unedited_two_drop_copy_passes_every_pin():
    from oracle import two_drop
    mod = _two_drop_module(open(two_drop.__file__).read())
    failed = [name for name, ok in _two_drop_pins(mod) if not ok]
    assert not failed, failed


@pytest.mark.parametrize("what,old,new", TWO_DROP_MUTANTS, ids=[m[0] for m in TWO_DROP_MUTANTS])
def test_planted_two_drop_mistake_fails_a_pin(what, old, new):
    from oracle import two_drop
    text = open(two_drop.__file__).read()
    assert old in text, f"the text to edit is not in the two-drop oracle: {old}"
    caught = [name for name, ok in _two_drop_pins(_two_drop_module(text.replace(old, new, 1)), True) if not ok]
    print(what, "->", caught)
    assert caught, f"no pin catches: {what}"


# Slips in the four-delta and on-surface parts of ers_oracle.c, against the pins of
# test_oracle_four_delta.py and test_oracle_sharp.py (cheapest first, stopping at the first
# failure).
EXTRA_MUTANTS = [
    ("I4: coefficient of lambda^4 in the polynomial 4 -> 2",
     "((3.0 - 2.0 * l2 + 4.0 * l2 * l2) * exp(-l2)", "((3.0 - 2.0 * l2 + 2.0 * l2 * l2) * exp(-l2)"),
    ("I4: power of lambda in the erfc term 5 -> 4",
     "- 4.0 * l2 * l2 * l * erfc(l));", "- 4.0 * l2 * l2 * erfc(l));"),
    ("four deltas: rho_k^3 instead of rho_k^5 in the I4 column",
     "if (K == 4) A[k][3] = r * r * r * r * r * ora_I4(lam);", "if (K == 4) A[k][3] = r * r * r * ora_I4(lam);"),
    ("s#1: sign of the polynomial term",
     "double s1 = e + c / 3.0 * (5.0 * t - 2.0 * t * t2) * g;", "double s1 = e - c / 3.0 * (5.0 * t - 2.0 * t * t2) * g;"),
    ("on-surface double layer: sign of the stresslet",
     "for (int i = 0; i < 3; ++i) acc[i] += -6.0 * d[i] * dq * dn * k5 * w;",
     "for (int i = 0; i < 3; ++i) acc[i] += 6.0 * d[i] * dq * dn * k5 * w;"),
    ("s#3: coefficient 6 -> 4",
     "double s3 = e - c / 9.0 * (9.0 * t + 6.0 * t * t2 - 4.0 * t * t2 * t2) * g;",
     "double s3 = e - c / 9.0 * (9.0 * t + 4.0 * t * t2 - 4.0 * t * t2 * t2) * g;"),
    ("s#2: coefficient 14 -> 12",
     "double s2 = e - c / 3.0 * (3.0 * t - 14.0 * t * t2 + 4.0 * t * t2 * t2) * g;",
     "double s2 = e - c / 3.0 * (3.0 * t - 12.0 * t * t2 + 4.0 * t * t2 * t2) * g;"),
]


def _extra_pins():
    import test_oracle_four_delta as F
    import test_oracle_sharp as S
    # properties that fix the functions independently of their printed formulas first; the
    # 50-digit evaluation of those formulas last
    checks = [("I4 derivative and limits", F.test_I4_derivative_and_limits),
              ("four-delta weights at b = 0", lambda: F.test_weights_at_b0_are_the_exact_rationals((3, 4, 5, 6))),
              ("s# limits", S.test_sigma_sharp_limits),
              ("on-surface single layer, fifth order", S.test_on_surface_single_layer_fifth_order),
              ("on-surface self-convergence and agreement with extrapolation",
               S.test_on_surface_self_convergence_and_agreement_with_extrapolation),
              ("four deltas converge faster than three", F.test_four_deltas_converge_faster_than_three),
              ("s# against 50-digit values", S.test_sigma_sharp_against_mpmath)]
    for name, fn in checks:
        try:
            fn()
        except AssertionError:
            return [(name, False)]
    return [(name, True) for name, _ in checks]


@pytest.mark.parametrize("what,old,new", EXTRA_MUTANTS, ids=[m[0] for m in EXTRA_MUTANTS])
def test_planted_four_delta_or_sharp_mistake_fails_a_pin(tmp_path, what, old, new):
    pytest.importorskip("mpmath")
    text = open(SRC).read()
    assert old in text, f"the text to edit is not in the oracle: {old}"
    lib = _compile(tmp_path, "mutant", text.replace(old, new, 1))
    saved = oracle._lib
    oracle._lib = lib
    try:
        caught = [name for name, ok in _extra_pins() if not ok]
    finally:
        oracle._lib = saved
    print(what, "->", caught)
    assert caught, f"no pin catches: {what}"


def test_unedited_copy_passes_the_four_delta_and_sharp_pins(tmp_path):
    pytest.importorskip("mpmath")
    lib = _compile(tmp_path, "unedited", open(SRC).read())
    saved = oracle._lib
    oracle._lib = lib
    try:
        failed = [name for name, ok in _extra_pins() if not ok]
    finally:
        oracle._lib = saved
    assert not failed, failed


# Slips in the learned closure's parts of the oracle: the reduced one- and two-delta sums of
# ers_oracle.c, and the frame, curvatures, jets and targets of oracle/closure.py, against the pins
# of test_oracle_closure.py (cheapest first, stopping at the first failure).
CLOSURE_C_MUTANTS = [
    ("two-delta weights: sign of beta_1", "beta[1] = -a[0] / det;", "beta[1] = a[0] / det;"),
    ("gamma: rho^2 instead of rho^3", "c[k] = rho[k] * rho[k] * rho[k] * ora_I2(lam);",
     "c[k] = rho[k] * rho[k] * ora_I2(lam);"),
    ("reduced double layer: chi q(x0) dropped", "vv += beta[k] * (sv[k][i] * inv8pi + chi * qm0[i]);",
     "vv += beta[k] * (sv[k][i] * inv8pi);"),
    ("reduced sums: the sum of delta_k taken with delta_{k+1}",
     "double delta = rho[k] * h;\n                ora_sl_term(d, r, delta, tc, g, w[j], su[k], 0);",
     "double delta = rho[k + 1] * h;\n                ora_sl_term(d, r, delta, tc, g, w[j], su[k], 0);"),
]

CLOSURE_PY_MUTANTS = [
    ("principal frame: the eigenvector of k2 taken as t1", "v = evecs[:, 1]", "v = evecs[:, 0]"),
    ("principal frame: t2 = t1 x n0 (left-handed frame)", "t2 = np.cross(E[2], t1)", "t2 = np.cross(t1, E[2])"),
    ("shape operator: multiplied by |grad F| instead of divided",
     "S = (E[:2] @ hess @ E[:2].T) / np.linalg.norm(grad)", "S = (E[:2] @ hess @ E[:2].T) * np.linalg.norm(grad)"),
    ("jets: the factorials i! j! dropped", "return coef * fact[:, None]", "return coef"),
    ("jets: eta taken along t1", "eta = d[sel] @ frame[1] / h", "eta = d[sel] @ frame[0] / h"),
    ("correction: sign of the two-delta term", "outs.append(ur - gamma[:, None] * corr if ndelta == 2 else ur + corr)",
     "outs.append(ur + gamma[:, None] * corr if ndelta == 2 else ur + corr)"),
    ("targets: h^p of the single layer also for the double layer", "        p = 1 if layer == 0 else 0\n        S = scale",
     "        p = 1\n        S = scale"),
]


def _closure_pins(stop_at_failure=True):
    import test_oracle_closure as C
    checks = [("two-delta weights exact at b = 0", lambda: C.test_two_delta_weights_exact_at_zero((2.0, 3.0, 4.0))),
              ("two-delta weight identities", C.test_two_delta_weights_identities),
              ("plain sums beyond the reduced radius", C.test_targets_beyond_the_reduced_radius_take_the_plain_sums),
              ("sphere frame", C.test_sphere_frame_and_curvatures),
              ("ellipsoid axis points", C.test_ellipsoid_axis_points),
              ("principal directions and curvatures", C.test_ellipsoid_principal_directions_and_curvatures),
              ("exact fit of tangent polynomials", C.test_jets_exact_for_a_polynomial_in_the_tangent_coordinates),
              ("jets against Monge-patch derivatives", C.test_jets_match_surface_derivatives_on_the_sphere),
              ("targets and correction inverse", C.test_targets_and_apply_are_inverse),
              ("u2 - gamma c2 = u3", C.test_two_delta_value_with_three_delta_c2_is_the_three_delta_value),
              ("orders of convergence", C.test_reduced_sums_converge_at_their_orders)]
    out = []
    for name, fn in checks:
        try:
            fn()
            out.append((name, True))
        except (AssertionError, ValueError, TypeError, np.linalg.LinAlgError):
            out.append((name, False))
            if stop_at_failure:
                break
    return out


@pytest.mark.parametrize("what,old,new", CLOSURE_C_MUTANTS, ids=[m[0] for m in CLOSURE_C_MUTANTS])
def test_planted_reduced_sum_mistake_fails_a_pin(tmp_path, what, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, f"the text to edit is not unique in the oracle: {old}"
    lib = _compile(tmp_path, "mutant", text.replace(old, new, 1))
    saved = oracle._lib
    oracle._lib = lib
    try:
        caught = [name for name, ok in _closure_pins() if not ok]
    finally:
        oracle._lib = saved
    print(what, "->", caught)
    assert caught, f"no pin catches: {what}"


@pytest.mark.parametrize("what,old,new", CLOSURE_PY_MUTANTS, ids=[m[0] for m in CLOSURE_PY_MUTANTS])
def test_planted_closure_feature_mistake_fails_a_pin(what, old, new):
    import types

    import test_oracle_closure as C
    from oracle import closure
    text = open(closure.__file__).read()
    assert text.count(old) == 1, f"the text to edit is not unique in the closure oracle: {old}"
    mod = types.ModuleType("closure_copy")
    mod.__file__ = closure.__file__
    exec(compile(text.replace(old, new, 1), closure.__file__, "exec"), mod.__dict__)
    saved = C.closure
    C.closure = mod
    try:
        caught = [name for name, ok in _closure_pins() if not ok]
    finally:
        C.closure = saved
    print(what, "->", caught)
    assert caught, f"no pin catches: {what}"


def test_unedited_closure_oracle_passes_every_pin(tmp_path):
    lib = _compile(tmp_path, "unedited", open(SRC).read())
    saved = oracle._lib
    oracle._lib = lib
    try:
        failed = [name for name, ok in _closure_pins(False) if not ok]
    finally:
        oracle._lib = saved
    assert not failed, failed
