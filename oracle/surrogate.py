"""CPU oracle of the learned kernel surrogate: the network's forward and backward pass in FP64.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests use it to check the CUDA
training kernels' loss and gradient; the product never imports it.  It shares no code with the
CUDA path.

The network is the project's definition (the paper has none; the surrogate is a growth item of
the build): for inputs z = (z0, z1),

    a1 = W1 z + b1,   h1 = silu(a1)            (64 units)
    a2 = W2 h1 + b2,  h2 = silu(a2)            (64 units)
    a3 = W3 h2 + b3,  h3 = silu(a3)            (64 units)
    y  = w4 . h3 + b4
    L  = mean_s (y_s - t_s)^2

with silu(x) = x / (1 + exp(-x)).  The parameters enter every pass rounded to BF16 (round to
nearest, ties to even) and the derivative is taken with respect to those rounded values.
Parameter vector layout: W1[64][2], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], w4[64], b4.

Parity pins: the gradient against central finite differences of this same loss, and the BF16
rounding against torch's bfloat16 conversion (tests/test_surrogate_oracle.py).
"""
from __future__ import annotations

import numpy as np

H = 64
N_PARAM = 2 * H + H + H * H + H + H * H + H + H + 1   # 8577


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((b >> 16) & 1)
    r = ((b + bias) >> 16) << 16
    nan = np.isnan(np.asarray(x, np.float32))
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    return np.where(nan, np.float32(np.nan), out)


def unpack(w):
    """Split the parameter vector into (W1, b1, W2, b2, W3, b3, w4, b4) views."""
    w = np.asarray(w, np.float64)
    o = 0
    out = []
    for shape in ((H, 2), (H,), (H, H), (H,), (H, H), (H,), (H,), (1,)):
        n = int(np.prod(shape))
        out.append(w[o:o + n].reshape(shape))
        o += n
    assert o == N_PARAM
    return out


def _silu(x):
    return x / (1.0 + np.exp(-x))


def _silu_grad(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def forward(w, z):
    """Network output y for inputs z [n, 2] with parameters w (already rounded as the caller wants)."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(w)
    z = np.asarray(z, np.float64)
    h1 = _silu(z @ W1.T + b1)
    h2 = _silu(h1 @ W2.T + b2)
    h3 = _silu(h2 @ W3.T + b3)
    return h3 @ w4 + b4[0]


def loss_grad(w, z, t, round_bf16=True):
    """Loss mean((y - t)^2) and its gradient (FP64) at parameters w (BF16-rounded first unless told
    otherwise) for inputs z [n, 2] and targets t [n]."""
    wr = bf16_round(np.asarray(w, np.float32)).astype(np.float64) if round_bf16 else np.asarray(w, np.float64)
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(wr)
    z = np.asarray(z, np.float64)
    t = np.asarray(t, np.float64)
    n = len(t)
    a1 = z @ W1.T + b1
    h1 = _silu(a1)
    a2 = h1 @ W2.T + b2
    h2 = _silu(a2)
    a3 = h2 @ W3.T + b3
    h3 = _silu(a3)
    y = h3 @ w4 + b4[0]
    d = y - t
    loss = float(np.mean(d * d))
    dy = 2.0 * d / n
    g_w4 = h3.T @ dy
    g_b4 = np.array([dy.sum()])
    d3 = np.outer(dy, w4) * _silu_grad(a3)
    g_W3 = d3.T @ h2
    g_b3 = d3.sum(axis=0)
    d2 = (d3 @ W3) * _silu_grad(a2)
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * _silu_grad(a1)
    g_W1 = d1.T @ z
    g_b1 = d1.sum(axis=0)
    grad = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_W3.ravel(), g_b3, g_w4, g_b4])
    return loss, grad
