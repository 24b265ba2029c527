"""Pins of the oracle's smoothing functions, I0/I2 and the extrapolation solve (Sec. 2)."""
import json
import pathlib
import math
import os

import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")
mp.mp.dps = 50
GOLD = json.loads(pathlib.Path(os.path.join(os.path.dirname(__file__), "golden", "extrap_weights.json")).read_text())


def sigma_mp(t):
    """s_p(t)/t^p from Eqs. (s1)-(s3) at 50 digits."""
    t = mp.mpf(t)
    e, g, c = mp.erf(t), mp.exp(-t * t), 2 / mp.sqrt(mp.pi)
    s1 = e
    s2 = e - c * t * g
    s3 = e - c * (t + mp.mpf(2) / 3 * t**3) * g
    return [float(s1 / t), float(s2 / t**3), float(s3 / t**5)]


@pytest.mark.parametrize("t", [1e-6, 0.01, 0.2, 0.49999999, 0.5, 0.50000001, 0.8, 1.5, 3.0, 5.9, 6.0])
def test_sigma_matches_high_precision(t):
    got = oracle.sigma(t)
    ref = sigma_mp(t)
    for p in range(3):
        # series branch (t < 0.5): a few ulp; closed forms: cancellation in s_p, ~eps erf(t)/s_p(t)
        assert abs(got[p] - ref[p]) <= 1e-14 * abs(ref[p]), (p, got[p], ref[p])


def test_sigma_limits():
    c = 2 / math.sqrt(math.pi)
    got = oracle.sigma(0.0)
    assert np.allclose(got, [c, c * 2 / 3, c * 4 / 15], rtol=1e-15, atol=0)
    # s_p(t) -> 1: at t = 6 the deviation is below 1e-13 (Sec. 3.2 localizes at t > 6)
    t = 6.0
    sig = oracle.sigma(t)
    for p, pw in enumerate((1, 3, 5)):
        assert abs(sig[p] * t**pw - 1) < 1e-13


@pytest.mark.parametrize("lam", [0.0, 0.1, 0.7, 1.3, 2.5, 4.0])
def test_I0_I2_high_precision(lam):
    l = mp.mpf(lam)
    i0 = mp.exp(-l * l) / mp.sqrt(mp.pi) - l * mp.erfc(l)
    i2 = mp.mpf(2) / 3 * ((mp.mpf(1) / 2 - l * l) * mp.exp(-l * l) / mp.sqrt(mp.pi) + l**3 * mp.erfc(l))
    assert abs(oracle.I0(lam) - float(i0)) <= 1e-15 * max(1.0, abs(float(i0)))
    assert abs(oracle.I2(lam) - float(i2)) <= 1e-15 * max(1.0, abs(float(i2)))
    # even functions of lambda
    assert oracle.I0(-lam) == oracle.I0(lam) and oracle.I2(-lam) == oracle.I2(lam)


def test_I0_I2_values_and_derivative_identities():
    sp = math.sqrt(math.pi)
    assert abs(oracle.I0(0.0) - 1 / sp) < 1e-16
    assert abs(oracle.I2(0.0) - 1 / (3 * sp)) < 1e-16
    eps = 1e-5
    for lam in (0.3, 1.0, 2.0):
        d0 = (oracle.I0(lam + eps) - oracle.I0(lam - eps)) / (2 * eps)
        d2 = (oracle.I2(lam + eps) - oracle.I2(lam - eps)) / (2 * eps)
        assert abs(d0 + math.erfc(lam)) < 1e-9          # I0' = -erfc
        assert abs(d2 + 2 * lam * oracle.I0(lam)) < 1e-9  # I2' = -2 lambda I0


@pytest.mark.parametrize("case", GOLD["cases"])
def test_extrapolation_weights_at_zero_are_exact_rationals(case):
    rho = case["rho"]
    alpha = []
    for k in range(3):
        U = np.zeros((3, 1))
        U[k, 0] = 1.0
        out, rc = oracle.extrapolate(rho, 0.0, 1 / 32, U)
        assert rc == 0
        alpha.append(out[0])
    want = np.array(case["alpha_num"]) / case["alpha_den"]
    assert np.abs(np.array(alpha) - want).max() < 1e-12


@pytest.mark.parametrize("rho", [(2, 3, 4), (3, 4, 5)])
def test_extrapolation_recovers_model_value(rho):
    """U_k = u + c1 rho_k I0(b/delta_k) + c2 rho_k^3 I2(b/delta_k) returns u (Eq. (extrap_eqn))."""
    h = 1 / 64
    rng = np.random.default_rng(0)
    for b in rng.uniform(-4 * h, 4 * h, 20):
        u, c1, c2 = rng.standard_normal(3)
        U = np.array([[u + c1 * r * oracle.I0(b / (r * h)) + c2 * r**3 * oracle.I2(b / (r * h))] for r in rho])
        out, rc = oracle.extrapolate(rho, b, h, U)
        assert rc == 0 and abs(out[0] - u) < 1e-12 * (1 + abs(c1) + abs(c2))
    # weights sum to one at any b
    for b in (0.0, 0.01, -0.05, 0.2):
        out, _ = oracle.extrapolate(rho, b, h, np.ones((3, 1)))
        assert abs(out[0] - 1) < 1e-12
