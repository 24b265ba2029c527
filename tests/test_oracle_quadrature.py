"""Pins of the oracle's quadrature rule (Sec. 2.2) and closest-point search (Sec. 2)."""
import json
import pathlib
import os

import numpy as np
import pytest

import oracle
import workloads

GOLD = json.loads(pathlib.Path(os.path.join(os.path.dirname(__file__), "golden", "table1.json")).read_text())
SPHEROID = workloads.Shape(tuple(GOLD["shape"]["center"]), tuple(GOLD["shape"]["axes"]))


def ellipsoid_area(a, b, c):
    # Carlson's symmetric integral form of the ellipsoid surface area (independent of the rule).
    from scipy.special import elliprg
    return 4 * np.pi * a * b * c * elliprg(1 / a**2, 1 / b**2, 1 / c**2)


@pytest.mark.parametrize("k", range(4))
def test_node_counts_match_table1(k):
    inv = GOLD["inv_h"][k]
    x, n, w = oracle.quadrature(SPHEROID, 1.0 / inv)
    assert len(w) == GOLD["quads"][k]


@pytest.mark.parametrize("k", range(3))
def test_target_counts_match_table1(k):
    """Grid points (ih, jh, kh) with 0 <= b <= h; the 6 axis tips lie on the surface (b = 0)."""
    inv = GOLD["inv_h"][k]
    h = 1.0 / inv
    I = np.arange(-inv - 3, inv + 4)
    J = np.arange(-inv // 2 - 3, inv // 2 + 4)
    g = np.stack(np.meshgrid(I, J, J, indexing="ij"), -1).reshape(-1, 3).astype(float) * h
    _, _, b = oracle.closest_point(SPHEROID, g)
    assert int(((b >= 0) & (b <= h * (1 + 1e-12))).sum()) == GOLD["targets"][k]


def test_weights_integrate_area():
    for inv, tol in ((64, 5e-9), (128, 1e-12)):
        _, _, w = oracle.quadrature(workloads.unit_sphere(), 1.0 / inv)
        assert abs(w.sum() - 4 * np.pi) < tol
    for axes, inv, tol in (((1.0, 0.5, 0.5), 128, 1e-7), ((1.0, 0.8, 0.6), 128, 1e-8)):
        _, _, w = oracle.quadrature(workloads.Shape((0.0, 0.0, 0.0), axes), 1.0 / inv)
        assert abs(w.sum() - ellipsoid_area(*axes)) < tol


def test_quadrature_integrates_smooth_function():
    # integral of x1^2 over the unit sphere = 4 pi / 3
    x, _, w = oracle.quadrature(workloads.unit_sphere(), 1 / 64)
    assert abs((w * x[:, 0] ** 2).sum() - 4 * np.pi / 3) < 1e-8


def test_nodes_on_surface_with_unit_outward_normals():
    shape = workloads.Shape((0.1, -0.2, 0.05), (1.0, 0.8, 0.6))
    x, n, w = oracle.quadrature(shape, 1 / 32)
    c, a = np.array(shape.center), np.array(shape.axes)
    assert np.abs((((x - c) / a) ** 2).sum(1) - 1).max() < 1e-14
    assert np.abs(np.linalg.norm(n, axis=1) - 1).max() < 1e-14
    assert ((n * (x - c)).sum(1) > 0).all()
    assert (w >= 0).all()
    # lattice: two of the three coordinates are multiples of h
    on_lattice = (np.abs(x / (1 / 32) - np.round(x / (1 / 32))) < 1e-9).sum(1)
    assert (on_lattice >= 2).all()


@pytest.mark.parametrize("shape", [workloads.unit_sphere((0.2, 0.0, -0.1)),
                                   workloads.Shape((0.0, 0.0, 0.0), (1.0, 0.8, 0.6))])
def test_closest_point_recovers_construction(shape):
    rng = np.random.default_rng(3)
    y, x0g, n0g, bg = workloads.near_band_targets(shape, 500, 0.3, rng)
    x0, n0, b = oracle.closest_point(shape, y)
    assert np.abs(x0 - x0g).max() < 1e-13
    assert np.abs(n0 - n0g).max() < 1e-12
    assert np.abs(b - bg).max() < 1e-13


def test_closest_point_far_and_medial_targets_are_valid():
    shape = workloads.Shape((0.0, 0.0, 0.0), (1.0, 0.8, 0.6))
    rng = np.random.default_rng(4)
    y = rng.uniform(-2, 2, (2000, 3))
    y[:5, 2] = 0.0  # on a symmetry plane through the smallest axis
    y[:5] *= 0.2
    x0, n0, b = oracle.closest_point(shape, y)
    a = np.array(shape.axes)
    assert np.abs(((x0 / a) ** 2).sum(1) - 1).max() < 1e-12
    assert np.abs(np.linalg.norm(y - x0, axis=1) - np.abs(b)).max() < 1e-13
    # no surface sample is closer than the reported distance
    xs, _, _ = oracle.quadrature(shape, 1 / 32)
    dmin = np.sqrt(((y[:, None, :] - xs[None, :, :]) ** 2).sum(-1)).min(1)
    assert (np.abs(b) <= dmin + 1e-12).all()
    inside = ((y / a) ** 2).sum(1) < 1
    assert ((b < 0) == inside).all()
