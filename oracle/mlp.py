"""FP64 oracle of the surrogate network (test infrastructure only).

A 4 -> 64 -> 64 -> 2 multilayer perceptron with exact (erf) GELU hidden
activations, weights rounded to bfloat16 before use (round to nearest even),
inputs and outputs standardised with stored means and deviations, mean
squared error on the standardised outputs, and Adam on float master weights.
Plain numpy in float64; no code shared with the CUDA kernels.

Parameter vector layout (4610 values): W1[64,4], b1[64], W2[64,64], b2[64],
W3[2,64], b3[2], each row-major (out, in).
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

IN, HID, OUT = 4, 64, 2
SHAPES = [(HID, IN), (HID,), (HID, HID), (HID,), (OUT, HID), (OUT,)]
NPARAM = sum(int(np.prod(s)) for s in SHAPES)


def bf16_round(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    nan = np.isnan(a)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def unpack(p):
    p = np.asarray(p, np.float64)
    out, k = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(p[k:k + n].reshape(s))
        k += n
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, Xn, round_bf16=True):
    """Standardised inputs (n, 4) -> standardised outputs (n, 2) and the cache.
    The weights are used rounded to bfloat16 unless round_bf16 is False."""
    if round_bf16:
        W1, b1, W2, b2, W3, b3 = [bf16_round(w) for w in unpack(np.asarray(params, np.float32))]
    else:
        W1, b1, W2, b2, W3, b3 = unpack(params)
    Z1 = Xn @ W1.T + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2.T + b2
    H2 = gelu(Z2)
    Y = H2 @ W3.T + b3
    return Y, (Xn, Z1, H1, Z2, H2, W2, W3)


def loss_grad(params, Xn, Tn, round_bf16=True):
    """Mean squared error over n samples and 2 outputs, and its gradient with
    respect to the (bfloat16-rounded) parameters, by the chain rule."""
    Y, (X, Z1, H1, Z2, H2, W2, W3) = forward(params, Xn, round_bf16)
    n = X.shape[0]
    E = Y - Tn
    loss = float((E * E).sum() / (n * OUT))
    D3 = 2.0 * E / (n * OUT)
    gW3 = D3.T @ H2
    gb3 = D3.sum(0)
    D2 = (D3 @ W3) * gelu_grad(Z2)
    gW2 = D2.T @ H1
    gb2 = D2.sum(0)
    D1 = (D2 @ W2) * gelu_grad(Z1)
    gW1 = D1.T @ X
    gb1 = D1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction; t counts from 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


class Standardizer:
    def __init__(self, X, Y):
        self.mx, self.sx = X.mean(0), X.std(0) + 1e-12
        self.my, self.sy = Y.mean(0), Y.std(0) + 1e-12

    def x(self, X):
        return (X - self.mx) / self.sx

    def y(self, Y):
        return (Y - self.my) / self.sy

    def y_inv(self, Yn):
        return Yn * self.sy + self.my
