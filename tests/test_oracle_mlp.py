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


def test_gelu_at_normal_cdf_table_values():
    """GELU(z) = z Phi(z), Phi the standard normal distribution function (textbook values)."""
    for z, phi in ((0.0, 0.5), (1.0, 0.8413447460685429), (-1.0, 0.15865525393145707), (0.5, 0.6914624612740131),
                   (2.0, 0.9772498680518208), (-2.0, 0.022750131948179195)):
        assert abs(mlp.gelu(np.array([z]))[0] - z * phi) <= 1e-15


def test_forward_of_a_hand_built_network():
    """One path through the layers with weights chosen so that every pre-activation equals 1:
    input x_5 = 1 -> W1[7, 5] = 1 -> GELU(1) = Phi(1) -> W2[3, 7] = 1/Phi(1) -> ... -> W4[2, 11] =
    2/Phi(1), b4 = (0.25, -0.5, 0.75): outputs (0.25, -0.5, 2.75); every other weight is zero, and
    the hidden biases of the other units are -1 so that their GELU is -Phi(-1) (which the zero
    weights of the next layer ignore).  Pins the layer order, the [out][in] weight layout and the
    bias of each layer, unquantized."""
    phi1 = 0.8413447460685429
    d = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    d["W1"][7, 5] = 1.0
    d["W2"][3, 7] = 1.0 / phi1
    d["W3"][11, 3] = 1.0 / phi1
    d["W4"][2, 11] = 2.0 / phi1
    for b in ("b1", "b2", "b3"):
        d[b][:] = -1.0
    d["b1"][7], d["b2"][3], d["b3"][11] = 0.0, 0.0, 0.0
    d["b4"][:3] = (0.25, -0.5, 0.75)
    X = np.zeros((2, mlp.IN))
    X[0, 5] = 1.0
    y, c = mlp.forward(mlp.pack(d), X, quantize=False)
    assert np.allclose(y[0], [0.25, -0.5, 2.75], atol=1e-14, rtol=0)
    assert np.allclose(c["z3"][0, 11], 1.0, atol=1e-14) and np.allclose(c["a1"][0, 0], -0.15865525393145707, atol=1e-15)
    # the zero input: every path is cut at the first layer, so z2 = b2 (unit 3: 0, others: -1)
    assert np.allclose(y[1], [0.25, -0.5, 0.75 + 2.0 / phi1 * mlp.gelu(np.array([0.0]))[0]], atol=1e-14)
