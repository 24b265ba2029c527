"""FP64 CPU oracle (plain C, OpenMP over targets) for the extrapolated-regularization method.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may load this package; the GPU library never does, and this package never loads
the GPU library.  The C source is ``ers_oracle.c``; every function there cites the passage of
Siebor & Tlupova it follows.

Functions:
  quadrature(shape, h)                      Sec. 2.2 lattice-crossing nodes, normals, weights
  closest_point(shape, y)                   x0, n0, b with y = x0 + b n0 (Sec. 2)
  evaluate(nodes, f, q, y, cp, f0, q0, ...) SL and DL values, direct or localized (Secs. 2, 3.3)
  sigma(t), I0(lam), I2(lam), extrapolate   building blocks (Eqs. (s1)-(s3), (I0), (I2), (extrap_eqn))
  evaluate_reduced, reduced_weights         the learned closure's one- and two-delta sums
  closure (submodule)                       the closure's features: frame, curvatures, density jets
  evaluate_tree(...), tree_info, tree_weights, lagrange
                                            the treecode far field of Sec. 3.4 (ers_treecode.c)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ers_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "ers_treecode.c")]
_LIB_PATH = os.path.join(_HERE, "_build", "libers_oracle.so")
_lock = threading.Lock()
_lib = None

DIRECT = 0
LOCALIZED = 1
ON_SURFACE_TOL = 1e-12  # |b| <= tol * (largest semi-axis) counts as on the surface


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    stale = not os.path.exists(_LIB_PATH) or any(os.path.getmtime(_LIB_PATH) < os.path.getmtime(f) for f in _SRCS)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, *_SRCS, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(ctypes.CDLL(build()))
    return _lib


def bind(lib):
    """Declare the argument types of the oracle's C functions on a loaded library (the built
    oracle, or a copy compiled from edited source by the planted-mistake tests)."""
    P = ctypes.POINTER(ctypes.c_double)
    i64, dbl, cint = ctypes.c_int64, ctypes.c_double, ctypes.c_int
    lib.ora_quadrature.restype = i64
    lib.ora_quadrature.argtypes = [P, P, dbl, P, P, P]
    lib.ora_closest_point.restype = None
    lib.ora_closest_point.argtypes = [P, P, P, i64, dbl, P, P, P]
    lib.ora_sigma.restype = None
    lib.ora_sigma.argtypes = [dbl, P]
    lib.ora_sigma_sharp.restype = None
    lib.ora_sigma_sharp.argtypes = [dbl, P]
    lib.ora_eval_sharp.restype = i64
    lib.ora_eval_sharp.argtypes = [P, P, P, P, P, i64, P, P, P, P, P, P, i64, dbl, P, dbl, dbl, P, P]
    lib.ora_I0.restype = dbl
    lib.ora_I0.argtypes = [dbl]
    lib.ora_I2.restype = dbl
    lib.ora_I2.argtypes = [dbl]
    lib.ora_extrapolate.restype = cint
    lib.ora_extrapolate.argtypes = [P, dbl, dbl, P, cint, P]
    lib.ora_eval.restype = i64
    lib.ora_eval.argtypes = [P, P, P, P, P, i64, P, P, P, P, P, P, i64, dbl, P, dbl, cint, P, P]
    lib.ora_eval_k.restype = i64
    lib.ora_eval_k.argtypes = [cint, P, P, P, P, P, i64, P, P, P, P, P, P, i64, dbl, P, dbl, cint, P, P]
    lib.ora_I4.restype = dbl
    lib.ora_I4.argtypes = [dbl]
    lib.ora_extrapolate_k.restype = cint
    lib.ora_extrapolate_k.argtypes = [cint, P, dbl, dbl, P, cint, P]
    lib.ora_eval_one_delta.restype = None
    lib.ora_eval_one_delta.argtypes = [P, P, P, P, P, i64, P, P, P, P, P, P, i64, dbl, dbl, P, P]
    lib.ora_reduced_weights.restype = cint
    lib.ora_reduced_weights.argtypes = [cint, P, dbl, dbl, P, P]
    lib.ora_eval_reduced.restype = i64
    lib.ora_eval_reduced.argtypes = [cint, P, P, P, P, P, i64, P, P, P, P, P, P, i64, dbl, P, dbl, P, P, P]
    lib.ora_plain.restype = None
    lib.ora_plain.argtypes = [P, P, P, P, P, i64, P, i64, P, P]
    lib.ora_num_threads.restype = cint
    I = ctypes.POINTER(ctypes.c_int64)
    lib.ora_eval_tree.restype = i64
    lib.ora_eval_tree.argtypes = [cint, P, P, P, P, P, i64, P, P, P, P, P, P, i64, dbl, P, dbl, dbl, i64,
                                  cint, P, P, I]
    lib.ora_tree_info.restype = i64
    lib.ora_tree_info.argtypes = [P, i64, i64, i64, P, P, P, I, I, I, I, I, I]
    lib.ora_tree_weights.restype = i64
    lib.ora_tree_weights.argtypes = [P, P, P, P, P, i64, i64, cint, i64, P]
    lib.ora_lagrange.restype = None
    lib.ora_lagrange.argtypes = [cint, dbl, dbl, dbl, P]
    lib.ora_cheb_points.restype = None
    lib.ora_cheb_points.argtypes = [cint, P]
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().ora_num_threads())


def quadrature(shape, h: float):
    """Nodes (N,3), outward normals (N,3), weights (N) of the Sec. 2.2 rule."""
    lib = _load()
    c, a = _c(shape.center), _c(shape.axes)
    N = lib.ora_quadrature(_p(c), _p(a), float(h), None, None, None)
    x, n, w = np.empty((N, 3)), np.empty((N, 3)), np.empty(N)
    N2 = lib.ora_quadrature(_p(c), _p(a), float(h), _p(x), _p(n), _p(w))
    assert N2 == N
    return x, n, w


def closest_point(shape, y):
    """Closest point x0, outward normal n0 and signed distance b (negative inside)."""
    lib = _load()
    c, a, y = _c(shape.center), _c(shape.axes), _c(y).reshape(-1, 3)
    M = y.shape[0]
    x0, n0, b = np.empty((M, 3)), np.empty((M, 3)), np.empty(M)
    tol = ON_SURFACE_TOL * max(shape.axes)
    lib.ora_closest_point(_p(c), _p(a), _p(y), M, tol, _p(x0), _p(n0), _p(b))
    return x0, n0, b


def sigma(t: float) -> np.ndarray:
    out = np.empty(3)
    _load().ora_sigma(float(t), _p(out))
    return out


def sigma_sharp(t: float) -> np.ndarray:
    """s#_p(t)/t^p for p = 1, 3, 5 (the on-surface functions of Sec. 2.1)."""
    out = np.empty(3)
    _load().ora_sigma_sharp(float(t), _p(out))
    return out


def I0(lam: float) -> float:
    return float(_load().ora_I0(float(lam)))


def I2(lam: float) -> float:
    return float(_load().ora_I2(float(lam)))


def I4(lam: float) -> float:
    """The lambda-dependence of the delta^5 error term (four-delta variant; see ers_oracle.c)."""
    return float(_load().ora_I4(float(lam)))


def extrapolate(rho, b: float, h: float, U: np.ndarray):
    """Solve Eq. (extrap_eqn) for u given U (K, nrhs) = the values for delta_1..K (K = 3, or 4 for
    the O(delta^7) variant with the c3 rho^5 I4 term)."""
    U = _c(U)
    K, nrhs = U.shape
    out = np.empty(nrhs)
    if K == 3:
        rc = _load().ora_extrapolate(_p(_c(rho)), float(b), float(h), _p(U), nrhs, _p(out))
    else:
        rc = _load().ora_extrapolate_k(K, _p(_c(rho)), float(b), float(h), _p(U), nrhs, _p(out))
    return out, rc


def evaluate(x, n, w, f, q, y, x0, n0, b, f0, q0, h, rho, tc=6.0, mode=LOCALIZED):
    """SL value u and DL value v (M,3) at targets y with len(rho) = 3 deltas (Eq. (extrap_eqn)) or
    4 (the O(delta^7) variant); see ers_oracle.c:ora_eval_k."""
    lib = _load()
    x, n, w, f, q = map(_c, (x, n, w, f, q))
    y, x0, n0, b, f0, q0 = map(_c, (y, x0, n0, b, f0, q0))
    N, M = w.shape[0], b.shape[0]
    u, v = np.empty((M, 3)), np.empty((M, 3))
    rho = _c(rho)
    assert len(rho) in (3, 4)
    nfail = lib.ora_eval_k(len(rho), _p(x), _p(n), _p(w), _p(f), _p(q), N, _p(y), _p(x0), _p(n0), _p(b), _p(f0),
                           _p(q0), M, float(h), _p(rho), float(tc), int(mode), _p(u), _p(v))
    return u, v, int(nfail)


def evaluate_sharp(x, n, w, f, q, y, x0, n0, b, f0, q0, h, rho, tc=6.0, rho_sharp=3.0):
    """Targets on the surface (b == 0): one sum with the s#_p of Sec. 2.1 and delta# = rho_sharp h,
    no extrapolation; the others by the extrapolated method.  See ers_oracle.c:ora_eval_sharp."""
    lib = _load()
    x, n, w, f, q = map(_c, (x, n, w, f, q))
    y, x0, n0, b, f0, q0 = map(_c, (y, x0, n0, b, f0, q0))
    N, M = w.shape[0], b.shape[0]
    u, v = np.empty((M, 3)), np.empty((M, 3))
    nfail = lib.ora_eval_sharp(_p(x), _p(n), _p(w), _p(f), _p(q), N, _p(y), _p(x0), _p(n0), _p(b), _p(f0), _p(q0),
                               M, float(h), _p(_c(rho)), float(tc), float(rho_sharp), _p(u), _p(v))
    return u, v, int(nfail)


def evaluate_one_delta(x, n, w, f, q, y, x0, n0, b, f0, q0, delta, tc=6.0):
    """Regularized sums u^delta, v^delta (Eqs. (Stokes_SL2), (Stokes_DL2)) for one delta."""
    lib = _load()
    x, n, w, f, q = map(_c, (x, n, w, f, q))
    y, x0, n0, b, f0, q0 = map(_c, (y, x0, n0, b, f0, q0))
    N, M = w.shape[0], b.shape[0]
    u, v = np.empty((M, 3)), np.empty((M, 3))
    lib.ora_eval_one_delta(_p(x), _p(n), _p(w), _p(f), _p(q), N, _p(y), _p(x0), _p(n0), _p(b), _p(f0), _p(q0), M,
                           float(delta), float(tc), _p(u), _p(v))
    return u, v


def reduced_weights(K: int, rho, b: float, h: float):
    """The one- or two-delta weights beta and gamma of the learned closure's reduced extrapolation
    (Eq. (extrap_eqn) with the c2 term kept aside); returns (beta (2,), gamma, rc)."""
    beta = np.empty(2)
    g = np.empty(1)
    rc = _load().ora_reduced_weights(int(K), _p(_c(rho)), float(b), float(h), _p(beta), _p(g))
    return beta, float(g[0]), int(rc)


def evaluate_reduced(K, x, n, w, f, q, y, x0, n0, b, f0, q0, h, rho, tc=6.0):
    """The learned closure's one-delta (K = 1) or two-delta (K = 2) sums by the definition, near
    radius tc rho[K-1] h; returns u, v (M,3) and gamma (M).  See ers_oracle.c:ora_eval_reduced."""
    lib = _load()
    x, n, w, f, q = map(_c, (x, n, w, f, q))
    y, x0, n0, b, f0, q0 = map(_c, (y, x0, n0, b, f0, q0))
    N, M = w.shape[0], b.shape[0]
    u, v, g = np.empty((M, 3)), np.empty((M, 3)), np.empty(M)
    assert K in (1, 2)
    lib.ora_eval_reduced(int(K), _p(x), _p(n), _p(w), _p(f), _p(q), N, _p(y), _p(x0), _p(n0), _p(b), _p(f0),
                         _p(q0), M, float(h), _p(_c(rho)), float(tc), _p(u), _p(v), _p(g))
    return u, v, g


def plain(x, n, w, f, q, y):
    """Unregularized, unsubtracted sums of Eqs. (Stokes_SL), (Stokes_DL)."""
    lib = _load()
    x, n, w, f, q, y = map(_c, (x, n, w, f, q, y))
    N, M = w.shape[0], y.shape[0]
    u, v = np.empty((M, 3)), np.empty((M, 3))
    lib.ora_plain(_p(x), _p(n), _p(w), _p(f), _p(q), N, _p(y), M, _p(u), _p(v))
    return u, v


# --- treecode far field (Sec. 3.4; ers_treecode.c) ---------------------------------------

def _pi(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def evaluate_tree(x, n, w, f, q, y, x0, n0, b, f0, q0, h, rho, tc=6.0, theta=0.6, n0_leaf=2000, p=6,
                  stats=False):
    """evaluate() with the far sums by the kernel-independent treecode (MAC theta, leaf size
    n0_leaf, degree p); stats=True also returns (M, 4) int64 per-target counts: clusters
    approximated, nodes in them, far pairs summed directly, near pairs."""
    lib = _load()
    x, n, w, f, q = map(_c, (x, n, w, f, q))
    y, x0, n0, b, f0, q0 = map(_c, (y, x0, n0, b, f0, q0))
    N, M = w.shape[0], b.shape[0]
    u, v = np.empty((M, 3)), np.empty((M, 3))
    st = np.zeros((M, 4), dtype=np.int64)
    rho = _c(rho)
    assert len(rho) in (3, 4) and 1 <= p <= 30
    nfail = lib.ora_eval_tree(len(rho), _p(x), _p(n), _p(w), _p(f), _p(q), N, _p(y), _p(x0), _p(n0), _p(b),
                              _p(f0), _p(q0), M, float(h), _p(rho), float(tc), float(theta), int(n0_leaf), int(p),
                              _p(u), _p(v), _pi(st))
    return (u, v, int(nfail), st) if stats else (u, v, int(nfail))


def tree_info(x, n0_leaf):
    """The octree of the treecode: dict of per-cluster arrays lo, hi (C,3), rc, start, count, level,
    nchild, parent (C,), and perm (N,) (the node order of the leaves)."""
    lib = _load()
    x = _c(x)
    N = x.shape[0]
    cap = max(64, 4 * N // max(1, int(n0_leaf)) + 64)
    while True:
        lo, hi = np.empty((cap, 3)), np.empty((cap, 3))
        rc = np.empty(cap)
        ints = [np.empty(cap, dtype=np.int64) for _ in range(5)]
        perm = np.empty(N, dtype=np.int64)
        nc = lib.ora_tree_info(_p(x), N, int(n0_leaf), cap, _p(lo), _p(hi), _p(rc), *map(_pi, ints), _pi(perm))
        if nc >= 0:
            break
        cap = -nc
    start, count, level, nchild, parent = (a[:nc] for a in ints)
    return dict(lo=lo[:nc], hi=hi[:nc], rc=rc[:nc], start=start, count=count, level=level, nchild=nchild,
                parent=parent, perm=perm)


def tree_weights(x, n, w, f, q, n0_leaf, p):
    """Modified weights of Eq. (mod_weights) of every cluster: (C, (p+1)^3, 15) with the densities
    f w (0:3), n w (3:6), q_j n_k w (6:15, index 6 + 3 j + k)."""
    lib = _load()
    x, n, w, f, q = map(_c, (x, n, w, f, q))
    N = x.shape[0]
    cap = max(64, 4 * N // max(1, int(n0_leaf)) + 64)
    nk = (p + 1) ** 3
    while True:
        W = np.empty((cap, nk, 15))
        nc = lib.ora_tree_weights(_p(x), _p(n), _p(w), _p(f), _p(q), N, int(n0_leaf), int(p), cap, _p(W))
        if nc >= 0:
            return W[:nc]
        cap = -nc


def lagrange(p, c, hw, xs):
    """Barycentric Lagrange basis at the p+1 Chebyshev points of [c - hw, c + hw], at each x in xs."""
    lib = _load()
    out = np.empty((len(xs), p + 1))
    buf = np.empty(p + 1)
    for i, xv in enumerate(xs):
        lib.ora_lagrange(int(p), float(c), float(hw), float(xv), _p(buf))
        out[i] = buf
    return out


def cheb_points(p):
    lib = _load()
    s = np.empty(p + 1)
    lib.ora_cheb_points(int(p), _p(s))
    return s
