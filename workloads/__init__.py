"""Seeded synthetic inputs for the extrapolated-regularization Stokes layer potentials.

This module is shared by the FP64 oracle tests, the GPU parity tests and the benchmark.  It
holds only input definitions: surface shapes, densities, target points and the random draws
behind them.  It contains none of the method's arithmetic (no quadrature, no kernels, no
closest-point search, no extrapolation).

Densities are polynomials of total degree <= 4 in (x1, x2, x3), one per vector component,
with i.i.d. N(0, 1) coefficients; on the unit sphere this space equals the spherical
harmonics of degree <= 4.  Near-band targets are built as y = x0 + b n0 from a surface
point x0 and its outward normal n0, so their closest point and signed distance are known by
construction (Sec. 2: y = x0 + b n with b the signed distance).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Monomials x1^i x2^j x3^k with i + j + k <= 4, in a fixed order (degree, then lexicographic).
MONOMIALS = [(i, j, d - i - j) for d in range(5) for i in range(d, -1, -1) for j in range(d - i, -1, -1)]
N_MONO = len(MONOMIALS)  # 35


@dataclasses.dataclass(frozen=True)
class Shape:
    """Ellipsoid sum(((x - center) / axes)^2) = 1; a sphere when all axes are equal."""

    center: tuple
    axes: tuple

    @property
    def is_sphere(self) -> bool:
        return self.axes[0] == self.axes[1] == self.axes[2]


def unit_sphere(center=(0.0, 0.0, 0.0)) -> Shape:
    return Shape(tuple(float(c) for c in center), (1.0, 1.0, 1.0))


def density_coeffs(rng: np.random.Generator) -> np.ndarray:
    """Coefficients (3, 35) of a degree <= 4 polynomial vector field."""
    return rng.standard_normal((3, N_MONO))


def poly_eval(coeffs: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Evaluate the polynomial vector field at points (M, 3) -> (M, 3), float64."""
    pts = np.asarray(pts, dtype=np.float64)
    out = np.zeros((pts.shape[0], 3))
    pw = [[np.ones(pts.shape[0])] for _ in range(3)]
    for a in range(3):
        for e in range(1, 5):
            pw[a].append(pw[a][-1] * pts[:, a])
    for m, (i, j, k) in enumerate(MONOMIALS):
        mono = pw[0][i] * pw[1][j] * pw[2][k]
        out += mono[:, None] * coeffs[:, m][None, :]
    return out


def poly_jacobian(coeffs: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Jacobian J[m, i, j] = d f_i / d x_j of the polynomial vector field at points (M, 3)."""
    pts = np.asarray(pts, dtype=np.float64)
    M = pts.shape[0]
    pw = [[np.ones(M)] for _ in range(3)]
    for a in range(3):
        for e in range(1, 5):
            pw[a].append(pw[a][-1] * pts[:, a])
    J = np.zeros((M, 3, 3))
    for m, ex in enumerate(MONOMIALS):
        for j in range(3):
            if ex[j] == 0:
                continue
            e = list(ex)
            e[j] -= 1
            d = ex[j] * pw[0][e[0]] * pw[1][e[1]] * pw[2][e[2]]
            J[:, :, j] += d[:, None] * coeffs[:, m][None, :]
    return J


def surface_points(shape: Shape, count: int, rng: np.random.Generator):
    """Random points x0 on the ellipsoid and their outward unit normals n0.

    The sphere uses normalised Gaussian directions (uniform on the sphere); an ellipsoid uses
    the parametric map with cos(theta) ~ U[-1, 1] and phi ~ U[0, 2 pi).
    """
    c = np.asarray(shape.center)
    a = np.asarray(shape.axes)
    if shape.is_sphere:
        v = rng.standard_normal((count, 3))
        n0 = v / np.linalg.norm(v, axis=1, keepdims=True)
        x0 = c + a[0] * n0
        return x0, n0
    ct = rng.uniform(-1.0, 1.0, count)
    st = np.sqrt(1.0 - ct * ct)
    ph = rng.uniform(0.0, 2.0 * math.pi, count)
    u = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)
    x0 = c + a * u
    g = u / a  # gradient direction of the implicit function
    n0 = g / np.linalg.norm(g, axis=1, keepdims=True)
    return x0, n0


def near_band_targets(shape: Shape, count: int, bmax: float, rng: np.random.Generator):
    """Targets y = x0 + b n0 with b ~ U[-bmax, bmax]; returns (y, x0, n0, b)."""
    x0, n0 = surface_points(shape, count, rng)
    b = rng.uniform(-bmax, bmax, count)
    y = x0 + b[:, None] * n0
    return y, x0, n0, b


def box_targets(count: int, half: float, rng: np.random.Generator, center=(0.0, 0.0, 0.0)):
    return np.asarray(center) + rng.uniform(-half, half, (count, 3))


@dataclasses.dataclass
class Workload:
    """One evaluation problem: a surface, two densities and the non-node targets.

    Node targets (every quadrature node, evaluated on the surface) are appended by whoever
    builds the nodes, because the nodes are an output of the quadrature rule, not an input.
    """

    name: str
    shape: Shape
    h: float
    rho: tuple
    f_coef: np.ndarray
    q_coef: np.ndarray
    extra_targets: np.ndarray  # (K, 3) near-band then far points
    band_x0: np.ndarray  # (B, 3) construction closest points of the near-band part
    band_n0: np.ndarray
    band_b: np.ndarray
    nodes_as_targets: bool = True
    cutoff_t: float = 6.0


def make_workload(name: str, shape: Shape, h: float, rho, seed: int, n_band: int, band_bmax: float,
                  n_far: int = 0, far_half: float = 2.0, nodes_as_targets: bool = True) -> Workload:
    rng = np.random.default_rng(seed)
    f_coef = density_coeffs(rng)
    q_coef = density_coeffs(rng)
    trng = np.random.default_rng(seed + 100)
    y_band, x0, n0, b = near_band_targets(shape, n_band, band_bmax, trng)
    far = box_targets(n_far, far_half, trng, shape.center) if n_far else np.zeros((0, 3))
    return Workload(name, shape, h, tuple(float(r) for r in rho), f_coef, q_coef,
                    np.concatenate([y_band, far], axis=0), x0, n0, b, nodes_as_targets)


def config(name: str) -> Workload:
    """The workloads of the evaluation, by name.

    sphere16    : unit sphere, h = 1/16, rho = (2,3,4); nodes + 2,000 band points |b| <= 4h.
    ellipsoid64 : ellipsoid (1, 0.8, 0.6), h = 1/64; nodes + 60,000 band points with
                  |b| <= 4 delta_3 (< 0.36, the smallest radius of curvature) + 20,000 points
                  uniform in [-2, 2]^3.
    sphere128   : unit sphere, h = 1/128 (N = 272,718); nodes + 100,000 band points
                  |b| <= 4h + 20,000 points uniform in [-2, 2]^3.
    sphere32    : unit sphere, h = 1/32; nodes + 2,000 band points (a mid-size parity case).
    sphere64    : unit sphere, h = 1/64; nodes + 25,000 band points + 5,000 box points (profiling).
    """
    if name == "sphere16":
        return make_workload(name, unit_sphere(), 1 / 16, (2, 3, 4), 1001, 2000, 4 / 16)
    if name == "sphere32":
        return make_workload(name, unit_sphere(), 1 / 32, (2, 3, 4), 1005, 2000, 4 / 32)
    if name == "sphere64":
        return make_workload(name, unit_sphere(), 1 / 64, (2, 3, 4), 1006, 25000, 4 / 64, n_far=5000)
    if name == "ellipsoid64":
        h = 1 / 64
        return make_workload(name, Shape((0.0, 0.0, 0.0), (1.0, 0.8, 0.6)), h, (2, 3, 4), 1002,
                             60000, 4 * 4 * h, n_far=20000)
    if name == "sphere128":
        return make_workload(name, unit_sphere(), 1 / 128, (2, 3, 4), 1003, 100000, 4 / 128,
                             n_far=20000)
    raise KeyError(name)


@dataclasses.dataclass
class BatchBody:
    """One surface of the batched workload with nrhs densities and its own targets."""

    shape: Shape
    h: float
    f_coefs: list
    q_coefs: list
    band: np.ndarray  # near-band targets added to the body's own nodes (may be empty)


def batched_config(gap: float = 0.01, nrhs: int = 8, n_bodies: int = 16, seed: int = 1004,
                   h_pair: float = 1 / 96):
    """Two unit spheres at (0,0,0) and (2 + gap, 0, 0) with spacing h_pair, each evaluated at the
    nodes of both (self and neighbour), plus n_bodies spheres/ellipsoids with semi-axes
    U[0.6, 1], spacing h in {1/32, 1/48, 1/64, 1/96} and centres 4 apart, each evaluated at its
    own nodes plus 5 % near-band points; nrhs seeded degree-4 densities per surface.
    Returns (pair, bodies): pair = [BatchBody, BatchBody], bodies = [BatchBody] * n_bodies."""
    rng = np.random.default_rng(seed)

    def dens():
        return [density_coeffs(rng) for _ in range(nrhs)], [density_coeffs(rng) for _ in range(nrhs)]

    pair = []
    for c in ((0.0, 0.0, 0.0), (2.0 + gap, 0.0, 0.0)):
        f, q = dens()
        pair.append(BatchBody(unit_sphere(c), h_pair, f, q, np.zeros((0, 3))))
    hs = [1 / 32, 1 / 48, 1 / 64, 1 / 96]
    bodies = []
    for i in range(n_bodies):
        axes = tuple(float(a) for a in rng.uniform(0.6, 1.0, 3))
        if i % 4 == 0:
            axes = (axes[0],) * 3
        center = (10.0 + 4.0 * (i % 4), 4.0 * (i // 4), 0.0)
        h = hs[int(rng.integers(0, len(hs)))]
        shape = Shape(center, axes)
        f, q = dens()
        bodies.append(BatchBody(shape, h, f, q, None))
    return pair, bodies


def subsample(count: int, total: int, seed: int) -> np.ndarray:
    """Seeded subset of target indices (sorted)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(total, size=min(count, total), replace=False))
