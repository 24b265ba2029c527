"""FP64 reference of the closure network (TEST INFRASTRUCTURE ONLY; shares no code with the GPU
library).

Network: x (16) -> 64 -> 64 -> 64 -> 16 (3 outputs used), GELU(z) = z/2 (1 + erf(z / sqrt 2))
after the three hidden layers.  With quantize=True the weight matrices, the input and the three
hidden activations are rounded to bfloat16 (round to nearest, ties to even) as the tensor-core
kernel stores them; the biases and all sums stay unrounded.  Loss L = (1/n) sum_s 1/2 |y_s - t_s|^2
over the 3 used outputs; the gradient passes through the rounding unchanged (straight-through).

Parameter layout (10448 values): W1 (64x16), b1 (64), W2 (64x64), b2 (64), W3 (64x64), b3 (64),
W4 (16x64), b4 (16); weights row-major [out][in].
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

IN, HID, OUT, USED = 16, 64, 16, 3
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (HID, HID)),
          ("b3", (HID,)), ("W4", (OUT, HID)), ("b4", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    out, off = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[off:off + k], dtype=np.float64).reshape(shape)
        off += k
    return out


def pack(d):
    return np.concatenate([d[name].reshape(-1) for name, _ in SHAPES])


def bf16(x):
    """Round to bfloat16 (8-bit significand), ties to even, via the float32 bit pattern."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_d(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(p, X, quantize=True):
    """Outputs (n, 3) and the intermediate values needed by backward()."""
    q = (lambda a: bf16(a)) if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    P = unpack(p)
    W = {k: (q(v) if k.startswith("W") else v) for k, v in P.items()}
    a0 = q(X)
    z1 = a0 @ W["W1"].T + W["b1"]
    a1 = q(gelu(z1))
    z2 = a1 @ W["W2"].T + W["b2"]
    a2 = q(gelu(z2))
    z3 = a2 @ W["W3"].T + W["b3"]
    a3 = q(gelu(z3))
    y = a3 @ W["W4"][:USED].T + W["b4"][:USED]
    return y, dict(W=W, a0=a0, a1=a1, a2=a2, a3=a3, z1=z1, z2=z2, z3=z3)


def loss_and_grad(p, X, T, quantize=True):
    """Loss and gradient with respect to the (unrounded) parameters."""
    y, c = forward(p, X, quantize)
    n = X.shape[0]
    e = y - T[:, :USED]
    loss = 0.5 * float((e * e).sum()) / n
    d4 = e / n
    W = c["W"]
    g = {}
    g["W4"] = np.zeros((OUT, HID))
    g["W4"][:USED] = d4.T @ c["a3"]
    g["b4"] = np.zeros(OUT)
    g["b4"][:USED] = d4.sum(0)
    d3 = (d4 @ W["W4"][:USED]) * gelu_d(c["z3"])
    g["W3"], g["b3"] = d3.T @ c["a2"], d3.sum(0)
    d2 = (d3 @ W["W3"]) * gelu_d(c["z2"])
    g["W2"], g["b2"] = d2.T @ c["a1"], d2.sum(0)
    d1 = (d2 @ W["W2"]) * gelu_d(c["z1"])
    g["W1"], g["b1"] = d1.T @ c["a0"], d1.sum(0)
    return loss, pack(g)
