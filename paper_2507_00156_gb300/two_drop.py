"""Two drops nearly touching in Stokes flow (Sec. 4.3): the interface velocity from the integral
equation (IE-2Surf), solved by GMRES (ers_gmres) over the library's evaluation.

With mu_0 = 1 and the 1/(8 pi) normalization of Eqs. (Stokes_SL), (Stokes_DL), at the nodes of
drop b:
    (lambda_b + 1) u_b - 2 sum_m (lambda_m - 1) DL_m[u_m] = -2 sum_m SL_m[[f]_m],
DL_b and SL_b at the drop's own nodes are principal values (b = 0, chi = 1/2) evaluated with the
modified functions s#_p of Sec. 2.1 (ERS_OPT_SHARP, delta# = rho_sharp h); at the other drop's
nodes they are the nearly singular integrals of the extrapolated method (delta = rho_k h).  The
double layer of the other drop needs u_m at the closest point, from ers_node_interp.  The jump
of the surface force is [f] = 2 gamma H n - grad_S gamma with gamma = 1 + (x_1 - x_c)^2 and H = 1
on the unit spheres centred at (0, 0, 0) and (2, 0, eps), eps = 1/16^3.
"""
from __future__ import annotations

import numpy as np

from . import LAYER_DL, LAYER_SL, PREC_FP64, Surface, gmres, node_interp, vec_axpby

EPS = 1.0 / 16 ** 3


def jump_force(x: np.ndarray, n: np.ndarray, xc: float) -> np.ndarray:
    """[f] = 2 gamma n - (I - n n) grad gamma, gamma = 1 + (x_1 - xc)^2, on a unit sphere (H = 1)."""
    gam = 1.0 + (x[:, 0] - xc) ** 2
    grad = np.zeros_like(x)
    grad[:, 0] = 2.0 * (x[:, 0] - xc)
    tang = grad - np.einsum("ij,ij->i", grad, n)[:, None] * n
    return 2.0 * gam[:, None] * n - tang


class TwoDrops:
    """The discretized Eq. (IE-2Surf) on the current CUDA device."""

    def __init__(self, h: float, eps: float = EPS, lam=(2.0, 2.0), rho=(3.0, 4.0, 5.0), rho_sharp: float = 3.0,
                 cutoff_t: float = 6.0, precision: int = PREC_FP64, tree=None):
        import torch
        self.h, self.lam, self.rho, self.rho_sharp, self.cutoff_t = h, lam, rho, rho_sharp, cutoff_t
        self.precision, self.tree = precision, tree
        self.centers = (np.array([0.0, 0.0, 0.0]), np.array([2.0, 0.0, eps]))
        self.s = [Surface(c, (1.0, 1.0, 1.0), h) for c in self.centers]
        self.x, self.n = [], []
        for s in self.s:
            x, n, _ = s.nodes()
            self.x.append(x)
            self.n.append(n)
        self.N = [s.N for s in self.s]
        dev = self.x[0].device
        self.zeros = [torch.zeros(N, dtype=torch.float64, device=dev) for N in self.N]
        # closest points of the nodes of drop b on drop m (b != m)
        self.cross = [self.s[1 - b].closest_point(self.x[b]) for b in range(2)]
        # [f] at the nodes of each drop and at the closest points on it of the other drop's nodes
        self.jump = []
        self.jump_cross = []
        for b in range(2):
            m = 1 - b
            xb, nb = self.x[b].cpu().numpy(), self.n[b].cpu().numpy()
            self.jump.append(torch.from_numpy(jump_force(xb, nb, self.centers[b][0])).to(dev))
            x0, n0, _ = (t.cpu().numpy() for t in self.cross[b])
            self.jump_cross.append(torch.from_numpy(jump_force(x0, n0, self.centers[m][0])).to(dev))
        self.tmp = [torch.empty((N, 3), dtype=torch.float64, device=dev) for N in self.N]
        self.q0 = [torch.empty((N, 3), dtype=torch.float64, device=dev) for N in self.N]
        self.matvecs = 0

    @property
    def n_unknowns(self) -> int:
        return 3 * (self.N[0] + self.N[1])

    def split(self, u):
        return u[:3 * self.N[0]].view(-1, 3), u[3 * self.N[0]:].view(-1, 3)

    def _eval(self, m, b, layers, f0=None, q0=None, out=None):
        """Layer of drop m at the nodes of drop b into out (N_b, 3)."""
        s = self.s[m]
        y = self.x[b]
        kw = dict(rho=self.rho, cutoff_t=self.cutoff_t, precision=self.precision, layers=layers, tree=self.tree)
        if layers == LAYER_SL:
            kw["u"] = out
        else:
            kw["v"] = out
        if m == b:  # own nodes: closest point = the node, b = 0, s#_p
            s.eval(y, f0, q0, x0=self.x[b], n0=self.n[b], b=self.zeros[b], sharp=True, rho_sharp=self.rho_sharp, **kw)
        else:
            x0, n0, bb = self.cross[b]
            s.eval(y, f0, q0, x0=x0, n0=n0, b=bb, **kw)
        return out

    def matvec(self, u, y):
        """y = A u for device vectors of length n_unknowns."""
        us, ys = self.split(u), self.split(y)
        for m in range(2):
            self.s[m].set_density(q=us[m])
        for b in range(2):
            m = 1 - b
            node_interp(self.s[m], us[m], self.cross[b][0], self.cross[b][1], out=self.q0[b])
            self._eval(b, b, LAYER_DL, q0=us[b], out=ys[b])
            self._eval(m, b, LAYER_DL, q0=self.q0[b], out=self.tmp[b])
            yb, tb = ys[b].view(-1), self.tmp[b].view(-1)
            vec_axpby(0.0, tb, -2.0 * (self.lam[b] - 1.0), yb)     # y_b = -2 (lam_b - 1) DL_b[u_b]
            vec_axpby(-2.0 * (self.lam[m] - 1.0), tb, 1.0, yb)     # ... - 2 (lam_m - 1) DL_m[u_m]
            vec_axpby(self.lam[b] + 1.0, us[b].reshape(-1), 1.0, yb)  # ... + (lam_b + 1) u_b
        self.matvecs += 1

    def rhs(self):
        """-2 sum_m SL_m[[f]_m] at the nodes of both drops."""
        import torch
        out = torch.empty(self.n_unknowns, dtype=torch.float64, device=self.x[0].device)
        os_ = self.split(out)
        for m in range(2):
            self.s[m].set_density(f=self.jump[m])
        for b in range(2):
            m = 1 - b
            self._eval(b, b, LAYER_SL, f0=self.jump[b], out=os_[b])
            self._eval(m, b, LAYER_SL, f0=self.jump_cross[b], out=self.tmp[b])
            vec_axpby(-2.0, self.tmp[b].view(-1), -2.0, os_[b].reshape(-1))
        return out

    def solve(self, tol: float = 1e-10, maxit: int = 100):
        """(u, iterations, relative residual, converged); u on device, drop 1 then drop 2."""
        b = self.rhs()
        return gmres(self.matvec, b, tol=tol, maxit=maxit)


def self_convergence(u_coarse, x_coarse, u_fine, x_fine):
    """Eq. (error_h) at the coarse nodes, which are nodes of the finer grid: (max |e_i|, L2 of
    Eq. (error_L2)) over the velocity components at the coarse nodes of both drops (host arrays
    per drop)."""
    errs = []
    for b in range(2):
        key = {tuple(p): i for i, p in enumerate(x_fine[b])}
        idx = np.array([key[tuple(p)] for p in x_coarse[b]])
        errs.append(u_coarse[b] - u_fine[b][idx])
    e = np.concatenate(errs).ravel()
    return float(np.abs(e).max()), float(np.sqrt((e ** 2).sum() / len(e)))
