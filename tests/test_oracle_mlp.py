"""Pins of the FP64 reference network used to check the closure kernels."""
import numpy as np
import pytest

import workloads
from oracle import mlp


def test_bf16_rounding_known_values():
    # 8 significand bits: 1 + 2^-7 is representable, 1 + 2^-8 is a tie (to even: 1), 1 + 3*2^-9 -> 1 + 2^-7
    x = np.array([1.0, 1 + 2.0**-7, 1 + 2.0**-8, 1 + 3 * 2.0**-8, 1 + 3 * 2.0**-9, -2.5, 0.0, 3.0e38])
    want = np.array([1.0, 1 + 2.0**-7, 1.0, 1 + 2.0**-6, 1 + 2.0**-7, -2.5, 0.0, 2.99e38])
    got = mlp.bf16(x)
    assert np.array_equal(got[:7], want[:7])
    assert abs(got[7] / 3.0e38 - 1) < 2.0**-8


def test_gradient_matches_finite_differences_unquantized():
    rng = np.random.default_rng(0)
    p = rng.standard_normal(mlp.NPARAM) * 0.2
    X = rng.standard_normal((7, 16))
    T = rng.standard_normal((7, 4))
    loss, g = mlp.loss_and_grad(p, X, T, quantize=False)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    # W4 rows 3..15 and b4[3..15] do not reach the loss
    off_w4 = 1024 + 64 + 4096 + 64 + 4096 + 64
    for i in idx:
        e = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += e
        pm[i] -= e
        fd = (mlp.loss_and_grad(pp, X, T, False)[0] - mlp.loss_and_grad(pm, X, T, False)[0]) / (2 * e)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
        if off_w4 + 3 * 64 <= i < off_w4 + 16 * 64 or i >= off_w4 + 16 * 64 + 3:
            assert g[i] == 0.0


def test_quantized_forward_is_near_unquantized():
    rng = np.random.default_rng(1)
    p = rng.standard_normal(mlp.NPARAM) * 0.2
    X = rng.standard_normal((50, 16))
    yq, _ = mlp.forward(p, X, True)
    y, _ = mlp.forward(p, X, False)
    assert np.abs(yq - y).max() < 0.05 * np.abs(y).max()
    assert np.abs(yq - y).max() > 0.0


def test_poly_jacobian_matches_finite_differences():
    rng = np.random.default_rng(2)
    c = workloads.density_coeffs(rng)
    x = rng.uniform(-1, 1, (20, 3))
    J = workloads.poly_jacobian(c, x)
    for j in range(3):
        e = np.zeros(3)
        e[j] = 1e-6
        fd = (workloads.poly_eval(c, x + e) - workloads.poly_eval(c, x - e)) / 2e-6
        assert np.abs(fd - J[:, :, j]).max() < 1e-6
