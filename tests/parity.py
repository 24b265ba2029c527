"""Helpers that run the same seeded problem through the GPU library and through the oracle.

Each side builds its own nodes, closest points and densities; only the workload definition
(shape, h, rho, polynomial coefficients, non-node targets) is shared.  Node targets are each
side's own nodes, which the quadrature parity test shows to be the same array.
"""
import functools

import numpy as np

import oracle
import workloads


def rel_err(got, ref):
    """max_y |got - ref|_inf / max_y |ref|_inf (one number per layer)."""
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def per_target_rel_err(got, ref, floor=1e-3):
    """max over targets y of |got(y) - ref(y)|_inf / max(|ref(y)|_inf, floor max_y |ref(y)|_inf):
    each target against its own magnitude, with a floor of 1e-3 of the largest so that targets
    where the value nearly vanishes do not turn rounding into an unbounded relative error."""
    num = np.abs(got - ref).max(axis=1)
    den = np.maximum(np.abs(ref).max(axis=1), floor * np.abs(ref).max())
    return float((num / den).max())


@functools.lru_cache(maxsize=8)
def oracle_problem(name):
    wl = workloads.config(name)
    x, n, w = oracle.quadrature(wl.shape, wl.h)
    f = workloads.poly_eval(wl.f_coef, x)
    q = workloads.poly_eval(wl.q_coef, x)
    return wl, x, n, w, f, q


def oracle_eval_sharp(name, sel=None, rho_sharp=3.0, tc=6.0):
    """The oracle with the on-surface s# path (Sec. 2.1) for targets with b = 0."""
    wl, x, n, w, f, q = oracle_problem(name)
    y = oracle_targets(wl, x, sel)
    x0, n0, b = oracle.closest_point(wl.shape, y)
    f0 = workloads.poly_eval(wl.f_coef, x0)
    q0 = workloads.poly_eval(wl.q_coef, x0)
    u, v, _ = oracle.evaluate_sharp(x, n, w, f, q, y, x0, n0, b, f0, q0, wl.h, wl.rho, tc, rho_sharp)
    return y, u, v, b


def oracle_targets(wl, x, sel=None):
    y = np.concatenate([x, wl.extra_targets]) if wl.nodes_as_targets else wl.extra_targets.copy()
    return y if sel is None else y[sel]


def oracle_eval(name, sel=None, rho=None, tc=6.0, mode=oracle.LOCALIZED):
    wl, x, n, w, f, q = oracle_problem(name)
    y = oracle_targets(wl, x, sel)
    x0, n0, b = oracle.closest_point(wl.shape, y)
    f0 = workloads.poly_eval(wl.f_coef, x0)
    q0 = workloads.poly_eval(wl.q_coef, x0)
    u, v, _ = oracle.evaluate(x, n, w, f, q, y, x0, n0, b, f0, q0, wl.h, rho or wl.rho, tc, mode)
    return y, u, v, b


class GpuProblem:
    """The same workload on the GPU library."""

    def __init__(self, name, wl=None):
        import torch

        import paper_2507_00156_gb300 as ers
        self.ers = ers
        self.wl = wl or workloads.config(name)
        self.s = ers.Surface(self.wl.shape.center, self.wl.shape.axes, self.wl.h)
        xd, nd, wd = self.s.nodes()
        self.x = xd.cpu().numpy()
        self.dev = xd.device
        f = workloads.poly_eval(self.wl.f_coef, self.x)
        q = workloads.poly_eval(self.wl.q_coef, self.x)
        self.s.set_density(torch.from_numpy(f).to(self.dev), torch.from_numpy(q).to(self.dev))

    def targets(self, sel=None):
        wl = self.wl
        y = np.concatenate([self.x, wl.extra_targets]) if wl.nodes_as_targets else wl.extra_targets.copy()
        return y if sel is None else y[sel]

    def prepare(self, y):
        """Device targets, closest points from the library, densities at them."""
        import torch
        yd = torch.from_numpy(np.ascontiguousarray(y)).to(self.dev)
        x0, n0, b = self.s.closest_point(yd)
        x0h = x0.cpu().numpy()
        f0 = torch.from_numpy(workloads.poly_eval(self.wl.f_coef, x0h)).to(self.dev)
        q0 = torch.from_numpy(workloads.poly_eval(self.wl.q_coef, x0h)).to(self.dev)
        return yd, x0, n0, b, f0, q0

    def eval(self, y, precision=0, rho=None, tc=6.0, layers=3, given_cp=False, **opts):
        import torch
        yd, x0, n0, b, f0, q0 = self.prepare(y)
        kw = dict(x0=x0, n0=n0, b=b) if given_cp else {}
        u, v = self.s.eval(yd, f0, q0, rho=rho or self.wl.rho, cutoff_t=tc, precision=precision, layers=layers,
                           **kw, **opts)
        torch.cuda.synchronize()
        return (None if u is None else u.cpu().numpy()), (None if v is None else v.cpu().numpy()), b.cpu().numpy()
