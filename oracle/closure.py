"""Features and training targets of the learned near-field closure, written plainly in numpy
(TEST INFRASTRUCTURE ONLY; shares no code with the GPU library, which never loads it).

The closure replaces the three-delta near sums of Eq. (extrap_eqn) by one or two of them and a
correction predicted from local data at the closest point x0 of each target y = x0 + b n0:

  geometry   lambda_0 = b / delta_0, the principal curvatures k1 >= k2 (times h) of the ellipsoid
             at x0 (outward normal, positive on convex surfaces), rho_0 and rho_1;
  frame      t1, t2, n0: t1, t2 the principal directions at x0, or, where the two curvatures agree
             to 1e-6 of their size (every point of a sphere), t1 = n0 x a / |n0 x a| with a = e_x
             (e_y when |n0_x| >= 0.9) and t2 = n0 x t1;
  jets       derivatives of the density (each of its components along t1, t2, n0) with respect to
             the tangent-plane coordinates (xi, eta) = ((x - x0).t1, (x - x0).t2) / h, taken from
             the least-squares polynomial of total degree <= 4 in (xi, eta) fitted to the node
             values within 3.5 h of x0: d^(i+j) / dxi^i deta^j = i! j! c_ij.  The single layer uses
             the orders 0..2 (18 values), the double layer the orders 1..3 (27 values; Q = q - q(x0)
             vanishes at x0); within a component the order is (0,0), (1,0), (0,1), (2,0), (1,1),
             (0,2), (3,0), (2,1), (1,2), (0,3), component-major;
  scale      S = the largest |jet| of the layer; the features are jets / S.

Why these jets: by Eq. (extrap_eqn) the near sums differ from the integral by c1 rho I0 +
c2 rho^3 I2 with c1, c2 fixed by the surface and the density near x0; the single-layer kernel is
O(1/r) and its delta^3 coefficient involves the density up to second derivatives, the
double-layer kernel is O(1/r^2) and involves one derivative more.  The coefficients are linear in
the density, so the closure predicts the linear map (a function of the geometry) and applies it
to the jets.

Targets (per layer, in the frame t1, t2, n0, divided by S h^p with p = 1 for the single layer and
p = 0 for the double layer):
  ndelta = 2: c2 = (u2 - u3) / gamma, u2 the two-delta value, u3 the three-delta method's value;
              sample weight (gamma / gamma(0))^2, or 0 where |gamma| < 0.01 |gamma(0)|;
  ndelta = 1: u3 - u1 (the whole correction of the single sum), weight 1.
A target takes no correction (scale 0, weight 0) when |b| exceeds the reduced near radius
tc rho_{K-1} h, when the fit has fewer than 15 nodes or is rank deficient, or when |lambda_0| > 64.
"""
from __future__ import annotations

import math

import numpy as np

FIT_RADIUS = 3.5  # in units of h
MONOMIALS = [(d - j, j) for d in range(5) for j in range(d + 1)]  # degree <= 4, (i, j) = xi^i eta^j
SL_ORDERS = (0, 2)
DL_ORDERS = (1, 3)
NGEOM = 5


def layer_monomials(layer: int):
    lo, hi = SL_ORDERS if layer == 0 else DL_ORDERS
    return [k for k, (i, j) in enumerate(MONOMIALS) if lo <= i + j <= hi]


def fallback_frame(n0):
    """t1 = n0 x a / |n0 x a| (a = e_x, or e_y when |n0_x| >= 0.9), t2 = n0 x t1; rows (t1, t2, n0)."""
    n0 = np.asarray(n0, dtype=np.float64)
    a = np.array([1.0, 0.0, 0.0]) if abs(n0[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    t1 = np.cross(n0, a)
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(n0, t1)
    return np.stack([t1, t2, n0])


def principal_frame(shape, x0, n0):
    """Rows (t1, t2, n0) and the principal curvatures (k1 >= k2) of the ellipsoid at x0.

    The shape operator of the level set F = sum ((x - c) / a)^2 = 1 on the tangent plane is
    P (Hess F) P / |grad F| with Hess F = diag(2 / a^2); its eigenvalues are the principal
    curvatures and its eigenvectors the principal directions.  t1 (the direction of k1) is signed so
    that its component along the fallback frame's first vector is >= 0 (along its second when that
    is 0)."""
    c = np.asarray(shape.center, dtype=np.float64)
    a = np.asarray(shape.axes, dtype=np.float64)
    p = np.asarray(x0, dtype=np.float64) - c
    grad = 2.0 * p / a**2
    hess = np.diag(2.0 / a**2)
    E = fallback_frame(n0)
    S = (E[:2] @ hess @ E[:2].T) / np.linalg.norm(grad)
    evals, evecs = np.linalg.eigh(S)  # ascending
    k1, k2 = float(evals[1]), float(evals[0])
    gap = math.hypot(S[0, 0] - S[1, 1], 2.0 * S[0, 1])
    if gap <= 1e-6 * (abs(S[0, 0]) + abs(S[1, 1])):
        return E, k1, k2
    v = evecs[:, 1]
    if v[0] < 0 or (v[0] == 0 and v[1] < 0):
        v = -v
    t1 = v[0] * E[0] + v[1] * E[1]
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(E[2], t1)
    return np.stack([t1, t2, E[2]]), k1, k2


def density_jets(x, vals, x0, frame, h):
    """Derivatives (15, 3) of the degree-4 least-squares fit of the node values (rows: MONOMIALS,
    columns: the components along t1, t2, n0) at x0, in units of h; None without a fit."""
    d = np.asarray(x, dtype=np.float64) - np.asarray(x0, dtype=np.float64)
    sel = (d * d).sum(axis=1) <= (FIT_RADIUS * h) ** 2
    if sel.sum() < len(MONOMIALS):
        return None
    xi = d[sel] @ frame[0] / h
    eta = d[sel] @ frame[1] / h
    V = np.stack([xi**i * eta**j for (i, j) in MONOMIALS], axis=1)
    if np.linalg.matrix_rank(V) < len(MONOMIALS):
        return None
    rhs = np.asarray(vals, dtype=np.float64)[sel] @ frame.T
    coef, *_ = np.linalg.lstsq(V, rhs, rcond=None)
    fact = np.array([math.factorial(i) * math.factorial(j) for (i, j) in MONOMIALS], dtype=np.float64)
    return coef * fact[:, None]


def features(shape, x, fvals, qvals, x0, n0, b, h, rho, ndelta, tc=6.0):
    """Per target: geometry (M, 5) = (lambda_0, k1 h, k2 h, rho_0, rho_1), frames (M, 3, 3), and per
    layer the scaled jets (M, J) and the scale S (M,) (0 = no correction)."""
    M = len(b)
    Rc = tc * rho[ndelta - 1] * h
    geom = np.zeros((M, NGEOM))
    frames = np.zeros((M, 3, 3))
    jets = [np.zeros((M, 3 * len(layer_monomials(0)))), np.zeros((M, 3 * len(layer_monomials(1))))]
    scale = np.zeros((M, 2))
    for m in range(M):
        fr, k1, k2 = principal_frame(shape, x0[m], n0[m])
        frames[m] = fr
        lam = b[m] / (rho[0] * h)
        geom[m] = (lam, k1 * h, k2 * h, rho[0], rho[1])
        ok = abs(b[m]) <= Rc and abs(lam) <= 64.0
        for layer, vals in ((0, fvals), (1, qvals)):
            if not ok:
                continue
            J = density_jets(x, vals, x0[m], fr, h)
            if J is None:
                continue
            jl = J[layer_monomials(layer)].T.reshape(-1)  # component-major
            S = float(np.abs(jl).max())
            if not (S > 0.0 and np.isfinite(S)):
                continue
            jets[layer][m] = jl / S
            scale[m, layer] = S
    return geom, frames, jets, scale


def gamma_at_zero(rho):
    """|gamma| at b = 0 of the two-delta weights: rho_0 rho_1 (rho_0 + rho_1) / (3 sqrt(pi))."""
    return rho[0] * rho[1] * (rho[0] + rho[1]) / (3.0 * math.sqrt(math.pi))


def targets(frames, scale, h, ndelta, u_red, v_red, gamma, u3, v3, rho):
    """Training targets (M, 3) per layer in the frame, and the sample weights (M,) per layer."""
    g0 = gamma_at_zero(rho)
    out, wts = [], []
    for layer, (ur, u3l) in enumerate(((u_red, u3), (v_red, v3))):
        p = 1 if layer == 0 else 0
        S = scale[:, layer]
        ok = S > 0
        if ndelta == 2:
            ok = ok & (np.abs(gamma) >= 0.01 * g0)
            c = np.where(ok[:, None], (ur - u3l) / np.where(ok, gamma, 1.0)[:, None], 0.0)
            w = np.where(ok, (gamma / g0) ** 2, 0.0)
        else:
            c = np.where(ok[:, None], u3l - ur, 0.0)
            w = ok.astype(np.float64)
        loc = np.einsum("mij,mj->mi", frames, c)
        den = np.where(ok, S * h**p, 1.0)
        out.append(np.where(ok[:, None], loc / den[:, None], 0.0))
        wts.append(w)
    return out, wts


def apply(frames, scale, h, ndelta, u_red, v_red, gamma, coef_s, coef_d):
    """The corrected values given the per-target correction coefficients c (M, 3) per layer in the
    frame (the network's output contracted with the jets): ndelta = 2: u = u2 - gamma S h^p (R c);
    ndelta = 1: u = u1 + S h^p (R c), R = [t1 t2 n0]."""
    outs = []
    for layer, (ur, c) in enumerate(((u_red, coef_s), (v_red, coef_d))):
        p = 1 if layer == 0 else 0
        corr = np.einsum("mij,mi->mj", frames, c) * (scale[:, layer] * h**p)[:, None]
        outs.append(ur - gamma[:, None] * corr if ndelta == 2 else ur + corr)
    return outs
