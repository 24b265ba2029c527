"""FP64 reference of the closure network (TEST INFRASTRUCTURE ONLY; shares no code with the GPU
library).

A sample record is XSTR = 48 values: the network input x = record[0:16] (the local geometry in
the first 5 entries, zeros after) and the density jets record[16:16 + nj] (nj = 18 for the single
layer, 27 for the double layer).

Network: x (16) -> 64 -> 64 -> 64 -> 96, GELU(z) = z/2 (1 + erf(z / sqrt 2)) after the three
hidden layers; the first 3 nj outputs are the coefficients A of a linear map from the jets to the
correction, c_e = sum_j A[e nj + j] jet_j (e = 0, 1, 2), evaluated unrounded.  With quantize=True
the weight matrices, the input x and the three hidden activations are rounded to bfloat16 (round
to nearest, ties to even) as the tensor-core kernel stores them; the biases and all sums stay
unrounded.  Loss L = (1/n) sum_s w_s/2 |c_s - t_s|^2 with the training record (t_s (3), w_s); the
gradient passes through the rounding unchanged (straight-through).

Parameter layout (15648 values): W1 (64x16), b1 (64), W2 (64x64), b2 (64), W3 (64x64), b3 (64),
W4 (96x64), b4 (96); weights row-major [out][in].
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

IN, HID, OUT = 16, 64, 96
JET_OFF, XSTR = 16, 48
NJ_SL, NJ_DL = 18, 27
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


def coefficients(p, X, nj, quantize=True):
    """The network's first 3 nj outputs A (n, 3 nj) for records X (n, XSTR), and the intermediate
    values needed by loss_and_grad()."""
    q = (lambda a: bf16(a)) if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    P = unpack(p)
    W = {k: (q(v) if k.startswith("W") else v) for k, v in P.items()}
    a0 = q(np.asarray(X, dtype=np.float64)[:, :IN])
    z1 = a0 @ W["W1"].T + W["b1"]
    a1 = q(gelu(z1))
    z2 = a1 @ W["W2"].T + W["b2"]
    a2 = q(gelu(z2))
    z3 = a2 @ W["W3"].T + W["b3"]
    a3 = q(gelu(z3))
    used = 3 * nj
    A = a3 @ W["W4"][:used].T + W["b4"][:used]
    return A, dict(W=W, a0=a0, a1=a1, a2=a2, a3=a3, z1=z1, z2=z2, z3=z3)


def forward(p, X, nj, quantize=True):
    """The correction c (n, 3) = A contracted with the jets of each record."""
    A, cache = coefficients(p, X, nj, quantize)
    jets = np.asarray(X, dtype=np.float64)[:, JET_OFF:JET_OFF + nj]
    c = np.einsum("nej,nj->ne", A.reshape(-1, 3, nj), jets)
    return c, cache


def loss_and_grad(p, X, T, nj, quantize=True):
    """Loss and gradient with respect to the (unrounded) parameters; T (n, 4) = (t (3), w)."""
    c, cache = forward(p, X, nj, quantize)
    n = X.shape[0]
    T = np.asarray(T, dtype=np.float64)
    w = T[:, 3]
    e = c - T[:, :3]
    loss = 0.5 * float((w[:, None] * e * e).sum()) / n
    jets = np.asarray(X, dtype=np.float64)[:, JET_OFF:JET_OFF + nj]
    d4 = ((w[:, None] * e)[:, :, None] * jets[:, None, :]).reshape(n, 3 * nj) / n  # dL/dA
    W = cache["W"]
    used = 3 * nj
    g = {}
    g["W4"] = np.zeros((OUT, HID))
    g["W4"][:used] = d4.T @ cache["a3"]
    g["b4"] = np.zeros(OUT)
    g["b4"][:used] = d4.sum(0)
    d3 = (d4 @ W["W4"][:used]) * gelu_d(cache["z3"])
    g["W3"], g["b3"] = d3.T @ cache["a2"], d3.sum(0)
    d2 = (d3 @ W["W3"]) * gelu_d(cache["z2"])
    g["W2"], g["b2"] = d2.T @ cache["a1"], d2.sum(0)
    d1 = (d2 @ W["W2"]) * gelu_d(cache["z1"])
    g["W1"], g["b1"] = d1.T @ cache["a0"], d1.sum(0)
    return loss, pack(g)
