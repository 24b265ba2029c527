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


@pytest.mark.parametrize("nj", [mlp.NJ_SL, mlp.NJ_DL])
def test_gradient_matches_finite_differences_unquantized(nj):
    rng = np.random.default_rng(0)
    p = rng.standard_normal(mlp.NPARAM) * 0.2
    X = np.zeros((7, mlp.XSTR))
    X[:, :5] = rng.standard_normal((7, 5))
    X[:, mlp.JET_OFF:mlp.JET_OFF + nj] = rng.standard_normal((7, nj))
    T = rng.standard_normal((7, 4))
    T[:, 3] = rng.uniform(0.0, 2.0, 7)
    T[2, 3] = 0.0  # a sample of weight 0 does not reach the loss
    loss, g = mlp.loss_and_grad(p, X, T, nj, quantize=False)
    off_w4 = 1024 + 64 + 4096 + 64 + 4096 + 64
    off_b4 = off_w4 + mlp.OUT * 64
    idx = np.concatenate([rng.choice(mlp.NPARAM, 50, replace=False),
                          off_w4 + 3 * nj * 64 + np.arange(3), [off_b4 + 3 * nj, off_b4 + 95]])
    for i in idx:
        e = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += e
        pm[i] -= e
        fd = (mlp.loss_and_grad(pp, X, T, nj, False)[0] - mlp.loss_and_grad(pm, X, T, nj, False)[0]) / (2 * e)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
        # W4 rows and b4 entries beyond the 3 nj coefficients do not reach the loss
        if off_w4 + 3 * nj * 64 <= i < off_b4 or i >= off_b4 + 3 * nj:
            assert g[i] == 0.0
    # the zero-weight sample: changing its target changes nothing
    T2 = T.copy()
    T2[2, :3] += 5.0
    assert mlp.loss_and_grad(p, X, T2, nj, False)[0] == loss


def test_quantized_forward_is_near_unquantized():
    rng = np.random.default_rng(1)
    p = rng.standard_normal(mlp.NPARAM) * 0.2
    X = np.zeros((50, mlp.XSTR))
    X[:, :5] = rng.standard_normal((50, 5))
    X[:, mlp.JET_OFF:mlp.JET_OFF + mlp.NJ_DL] = rng.standard_normal((50, mlp.NJ_DL))
    yq, _ = mlp.forward(p, X, mlp.NJ_DL, True)
    y, _ = mlp.forward(p, X, mlp.NJ_DL, False)
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
    input x_4 = 1 -> W1[7, 4] = 1 -> GELU(1) = Phi(1) -> W2[3, 7] = 1/Phi(1) -> ... -> W4[2, 11] =
    2/Phi(1), b4[:3] = (0.25, -0.5, 0.75): coefficients A[0:3] = (0.25, -0.5, 2.75); every other
    weight is zero, and the hidden biases of the other units are -1 so that their GELU is -Phi(-1)
    (which the zero weights of the next layer ignore).  With nj = 18 coefficient e nj + j multiplies
    jet j of component e: A[0], A[1], A[2] are component 0's weights of jets 0, 1, 2.  Pins the
    layer order, the [out][in] weight layout, the bias of each layer and the head's index order,
    unquantized."""
    phi1 = 0.8413447460685429
    nj = mlp.NJ_SL
    d = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    d["W1"][7, 4] = 1.0
    d["W2"][3, 7] = 1.0 / phi1
    d["W3"][11, 3] = 1.0 / phi1
    d["W4"][2, 11] = 2.0 / phi1
    for b in ("b1", "b2", "b3"):
        d[b][:] = -1.0
    d["b1"][7], d["b2"][3], d["b3"][11] = 0.0, 0.0, 0.0
    d["b4"][:3] = (0.25, -0.5, 0.75)
    d["b4"][nj + 1] = 10.0  # component 1, jet 1
    X = np.zeros((2, mlp.XSTR))
    X[0, 4] = 1.0
    X[:, mlp.JET_OFF:mlp.JET_OFF + 3] = (1.0, 2.0, 3.0)
    A, c = mlp.coefficients(mlp.pack(d), X, nj, quantize=False)
    assert np.allclose(A[0, :3], [0.25, -0.5, 2.75], atol=1e-14, rtol=0)
    assert np.allclose(c["z3"][0, 11], 1.0, atol=1e-14) and np.allclose(c["a1"][0, 0], -0.15865525393145707, atol=1e-15)
    y, _ = mlp.forward(mlp.pack(d), X, nj, quantize=False)
    assert np.allclose(y[0], [0.25 * 1 - 0.5 * 2 + 2.75 * 3, 10.0 * 2, 0.0], atol=1e-13, rtol=0)
    # the zero input: every path is cut at the first layer, so z2 = b2 (unit 3: 0, others: -1)
    a2 = 0.75 + 2.0 / phi1 * mlp.gelu(np.array([0.0]))[0]
    assert np.allclose(y[1], [0.25 * 1 - 0.5 * 2 + a2 * 3, 20.0, 0.0], atol=1e-13)
