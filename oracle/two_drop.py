"""FP64 CPU oracle of the two-drop problem of Sec. 4.3: the interface velocity u on two nearly
touching spherical drops from the integral equation (IE-2Surf), solved by GMRES.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU leg may
load this module; the GPU library never does.  It is written from the paper's statement of the
problem and builds on the oracle's evaluation (ers_oracle.c through ``oracle``).

With mu_0 = 1 and the normalization of Eqs. (Stokes_SL), (Stokes_DL) (the factor 1/(8 pi)),
Eq. (IE-2Surf) at the nodes x0 of drop b reads
    (lambda_b + 1) u_b(x0) - 2 sum_m (lambda_m - 1) DL_m[u_m](x0) = -2 sum_m SL_m[[f]_m](x0),
where DL_m at a node of its own drop (b = 0, chi = 1/2) is the principal value, evaluated with the
modified functions s#_p of Sec. 2.1 at delta# = 3h (``evaluate_sharp``), and DL_m at the nodes of
the other drop is the nearly singular integral, evaluated by the extrapolated method with
delta = 3h, 4h, 5h (``evaluate``).  [f] = 2 gamma H n - grad_S gamma with gamma = 1 + (x_1 -
x_c)^2, H = 1 (unit sphere, outward normal), grad_S gamma = (I - n n) grad gamma.  Drop 1 is centred
at the origin, drop 2 at (2, 0, eps), eps = 1/16^3.

Readings (the paper leaves them open):
  - the subtraction of Eq. (Stokes_DL1) for the other drop needs u_m at the closest point x0 on
    drop m, which is not a node: it is the value at x0 of the least-squares polynomial of total
    degree <= 4 in tangent-plane coordinates (xi, eta) = ((x - x0).t1, (x - x0).t2) / (3.5 h)
    fitted to u_m at the nodes of drop m within 3.5 h of x0 (an O(h^5) approximation, the order
    of the method);
  - GMRES without restart from u = 0, stopped when ||rhs - A u|| <= tol ||rhs||;
  - the error of Eq. (error_h) is taken at the nodes of the coarser grid, which are nodes of the
    finer one, on both drops; the max and the L2 norm of Eq. (error_L2) run over the 3N velocity
    components (with this reading the L2 error at h = 1/16 is 1.23e-4 against the 1.19e-4 of
    Table 2; over vector norms it would be 2.1e-4).
"""
from __future__ import annotations

import numpy as np

import oracle
import workloads

EPS = 1.0 / 16 ** 3
INTERP_RADIUS = 3.5  # in units of h
INTERP_DEG = 4


def surface_tension(x, xc):
    """gamma = 1 + (x_1 - x_c)^2 (Sec. 4.3)."""
    return 1.0 + (x[:, 0] - xc) ** 2


def jump_force(x, n, xc, H=1.0):
    """[f] = 2 gamma H n - grad_S gamma on a sphere of mean curvature H (Sec. 4.3)."""
    g = surface_tension(x, xc)
    grad = np.zeros_like(x)
    grad[:, 0] = 2.0 * (x[:, 0] - xc)
    grad_s = grad - (grad * n).sum(1)[:, None] * n
    return 2.0 * g[:, None] * H * n - grad_s


def tangent_basis(n0):
    """Orthonormal t1, t2 with n0 (M,3): t1 from the coordinate axis least aligned with n0."""
    k = np.argmin(np.abs(n0), axis=1)
    a = np.zeros_like(n0)
    a[np.arange(len(n0)), k] = 1.0
    t1 = a - (a * n0).sum(1)[:, None] * n0
    t1 /= np.linalg.norm(t1, axis=1)[:, None]
    t2 = np.cross(n0, t1)
    return t1, t2


def monomials(xi, eta, deg=INTERP_DEG):
    """xi^a eta^b with a + b <= deg, constant term first."""
    cols = [xi ** (d - b) * eta ** b for d in range(deg + 1) for b in range(d + 1)]
    return np.stack(cols, axis=-1)


def interp_weights(xm, x0, n0, h, radius=INTERP_RADIUS, deg=INTERP_DEG):
    """For each point x0 (on the surface with nodes xm): (node indices, weights) of the value at
    x0 of the least-squares polynomial fit described in the module docstring."""
    t1, t2 = tangent_basis(n0)
    out = []
    R = radius * h
    for i in range(len(x0)):
        d = xm - x0[i]
        r2 = (d * d).sum(1)
        idx = np.nonzero(r2 <= R * R)[0]
        xi = (d[idx] @ t1[i]) / R
        eta = (d[idx] @ t2[i]) / R
        Phi = monomials(xi, eta, deg)
        if len(idx) < Phi.shape[1]:
            raise ValueError("too few nodes for the local fit")
        # value at the origin = first coefficient = e_0^T pinv(Phi) u
        w = np.linalg.pinv(Phi)[0]
        out.append((idx, w))
    return out


def interp_apply(weights, vals):
    return np.stack([w @ vals[idx] for idx, w in weights])


def gmres(matvec, rhs, tol=1e-10, maxit=200):
    """GMRES (Saad & Schultz 1986) from x = 0 without restart: Arnoldi with modified
    Gram-Schmidt, the least-squares problem by Givens rotations.  Returns x, iterations and the
    relative residual."""
    n = rhs.size
    beta = np.linalg.norm(rhs)
    if beta == 0.0:
        return np.zeros(n), 0, 0.0
    V = np.zeros((maxit + 1, n))
    H = np.zeros((maxit + 1, maxit))
    cs, sn = np.zeros(maxit), np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    V[0] = rhs / beta
    k = 0
    rel = 1.0
    for k in range(maxit):
        w = matvec(V[k])
        for i in range(k + 1):
            H[i, k] = w @ V[i]
            w = w - H[i, k] * V[i]
        H[k + 1, k] = np.linalg.norm(w)
        if H[k + 1, k] > 0:
            V[k + 1] = w / H[k + 1, k]
        for i in range(k):  # previous rotations
            t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
            H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
            H[i, k] = t
        den = np.hypot(H[k, k], H[k + 1, k])
        cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
        H[k, k] = den
        H[k + 1, k] = 0.0
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        rel = abs(g[k + 1]) / beta
        if rel <= tol:
            break
    m = k + 1
    y = np.linalg.solve(np.triu(H[:m, :m]), g[:m])
    x = V[:m].T @ y
    return x, m, rel


class TwoDrops:
    """The discretized operator and right-hand side of Eq. (IE-2Surf) at spacing h."""

    def __init__(self, h, eps=EPS, lam=(2.0, 2.0), rho=(3.0, 4.0, 5.0), rho_sharp=3.0, tc=6.0):
        self.h, self.lam, self.rho, self.rho_sharp, self.tc = h, lam, rho, rho_sharp, tc
        self.centers = (np.array([0.0, 0.0, 0.0]), np.array([2.0, 0.0, eps]))
        self.shapes = [workloads.unit_sphere(tuple(c)) for c in self.centers]
        self.nodes = [oracle.quadrature(s, h) for s in self.shapes]  # (x, n, w) per drop
        self.N = [len(nd[2]) for nd in self.nodes]
        # closest points of every node on the other drop, and the interpolation there
        self.cross = []
        for b in range(2):
            m = 1 - b
            x0, n0, bb = oracle.closest_point(self.shapes[m], self.nodes[b][0])
            wts = interp_weights(self.nodes[m][0], x0, n0, h)
            self.cross.append((x0, n0, bb, wts))
        self.jump = [jump_force(nd[0], nd[1], c[0]) for nd, c in zip(self.nodes, self.centers)]

    def split(self, u):
        return u[:3 * self.N[0]].reshape(-1, 3), u[3 * self.N[0]:].reshape(-1, 3)

    def layer(self, m, b, f, q, layer):
        """SL (layer 0) or DL (layer 1) of densities f, q (node values of drop m) at the nodes of
        drop b, with the density at the closest point: f analytic ([f]), q interpolated."""
        x, n, w = self.nodes[m]
        y = self.nodes[b][0]
        zeros = np.zeros_like(x)
        fm = f if f is not None else zeros
        qm = q if q is not None else zeros
        if m == b:
            f0 = fm
            q0 = qm
            u, v, nf = oracle.evaluate_sharp(x, n, w, fm, qm, y, x, n, np.zeros(len(y)), f0, q0, self.h, self.rho,
                                             self.tc, self.rho_sharp)
        else:
            x0, n0, bb, wts = self.cross[b]
            f0 = jump_force(x0, n0, self.centers[m][0]) if f is not None else np.zeros_like(x0)
            q0 = interp_apply(wts, qm) if q is not None else np.zeros_like(x0)
            u, v, nf = oracle.evaluate(x, n, w, fm, qm, y, x0, n0, bb, f0, q0, self.h, self.rho, self.tc)
        assert nf == 0
        return u if layer == 0 else v

    def matvec(self, u):
        us = self.split(u)
        out = []
        for b in range(2):
            v = sum(2.0 * (self.lam[m] - 1.0) * self.layer(m, b, None, us[m], 1) for m in range(2))
            out.append((self.lam[b] + 1.0) * us[b] - v)
        return np.concatenate([o.ravel() for o in out])

    def rhs(self):
        out = []
        for b in range(2):
            out.append(-2.0 * sum(self.layer(m, b, self.jump[m], None, 0) for m in range(2)))
        return np.concatenate([o.ravel() for o in out])

    def solve(self, tol=1e-10, maxit=100):
        return gmres(self.matvec, self.rhs(), tol, maxit)


def self_convergence(u_coarse, nodes_coarse, u_fine, nodes_fine):
    """Eq. (error_h) at the coarse nodes (a subset of the fine ones): (max |e_i|, ||e||_2 of Eq.
    (error_L2)) over the velocity components at the coarse nodes of both drops."""
    errs = []
    for b in range(2):
        key = {tuple(p): i for i, p in enumerate(nodes_fine[b])}
        idx = np.array([key[tuple(p)] for p in nodes_coarse[b]])
        errs.append(u_coarse[b] - u_fine[b][idx])
    e = np.concatenate(errs).ravel()
    return float(np.abs(e).max()), float(np.sqrt((e ** 2).sum() / len(e)))
