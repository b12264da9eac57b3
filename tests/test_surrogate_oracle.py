"""Pins of the FP64 oracle of the kernel surrogate (oracle/surrogate.py).

* BF16 rounding against torch's own float32 -> bfloat16 conversion.
* The backward pass against central finite differences of the same loss (FP64).
* The loss returned with the gradient against a plain forward pass.
"""
import numpy as np
import pytest

from oracle import surrogate as so


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 2000), rng.normal(0, 1e4, 2000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 65504.0, 3.0e38]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(so.bf16_round(x).view(np.uint32), want.view(np.uint32))


def _random_problem(seed, n=48):
    rng = np.random.default_rng(seed)
    w = (rng.normal(0, 0.3, so.N_PARAM)).astype(np.float32)
    z = rng.uniform(-1, 1, (n, 2))
    t = rng.normal(0, 1, n)
    return w, z, t


def test_gradient_matches_finite_differences():
    w, z, t = _random_problem(1)
    w64 = w.astype(np.float64)
    _, g = so.loss_grad(w64, z, t, round_bf16=False)
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.choice(so.N_PARAM, 80, replace=False), [0, 127, 128, so.N_PARAM - 1]])
    eps = 1e-6
    for i in idx:
        wp, wm = w64.copy(), w64.copy()
        wp[i] += eps
        wm[i] -= eps
        lp, _ = so.loss_grad(wp, z, t, round_bf16=False)
        lm, _ = so.loss_grad(wm, z, t, round_bf16=False)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * (1 + abs(g[i])), (i, fd, g[i])


def test_loss_equals_forward_pass():
    w, z, t = _random_problem(3)
    loss, _ = so.loss_grad(w, z, t)
    y = so.forward(so.bf16_round(w).astype(np.float64), z)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-12)
