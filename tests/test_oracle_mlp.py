"""Pins of the surrogate-network oracle: bfloat16 rounding, GELU, forward,
gradients and Adam against independent references (PyTorch CPU float64
library routines, a textbook value, finite differences)."""

import math

import numpy as np
import pytest

from oracle import mlp
from workloads import surrogate as S

torch = pytest.importorskip('torch')


def test_bf16_rounding_ties_to_even_and_matches_library():
    one = 1.0
    assert mlp.bf16_round(np.float32(one))[()] == 1.0
    assert mlp.bf16_round(np.float32(1.0 + 2.0 ** -8))[()] == 1.0            # tie -> even
    assert mlp.bf16_round(np.float32(1.0 + 3 * 2.0 ** -8))[()] == 1.0 + 2.0 ** -6
    rng = np.random.default_rng(0)
    x = (rng.normal(0, 3, 100000) * 10.0 ** rng.integers(-8, 8, 100000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_gelu_textbook_values_and_derivative():
    # GELU(x) = x Phi(x); Phi(1) = 0.8413447460685429
    assert mlp.gelu(np.array(1.0)) == pytest.approx(0.8413447460685429, rel=1e-15)
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert mlp.gelu(np.array(10.0)) == pytest.approx(10.0, rel=1e-15)
    assert abs(mlp.gelu(np.array(-10.0))) < 1e-20
    z = np.linspace(-5, 5, 101)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, rtol=1e-8, atol=1e-10)
    assert mlp.gelu_grad(np.array(0.0)) == 0.5


def _torch_net(params):
    W1, b1, W2, b2, W3, b3 = [torch.tensor(w, dtype=torch.float64, requires_grad=True)
                              for w in mlp.unpack(params)]

    def f(X):
        h1 = torch.nn.functional.gelu(X @ W1.T + b1, approximate='none')
        h2 = torch.nn.functional.gelu(h1 @ W2.T + b2, approximate='none')
        return h2 @ W3.T + b3

    return f, [W1, b1, W2, b2, W3, b3]


def test_forward_and_gradient_match_pytorch_float64():
    rng = np.random.default_rng(1)
    p = S.init_params(3)[0]
    pr = mlp.bf16_round(p)                      # the weights the network uses
    X = rng.normal(0, 1, (257, 4))
    T = rng.normal(0, 1, (257, 2))
    Y, _ = mlp.forward(p, X)
    f, ws = _torch_net(pr)
    Xt = torch.tensor(X)
    Yt = f(Xt)
    assert np.allclose(Y, Yt.detach().numpy(), rtol=1e-12, atol=1e-12)
    loss_t = ((Yt - torch.tensor(T)) ** 2).mean()
    loss_t.backward()
    gt = np.concatenate([w.grad.numpy().ravel() for w in ws])
    loss, g = mlp.loss_grad(p, X, T)
    assert loss == pytest.approx(loss_t.item(), rel=1e-12)
    assert np.allclose(g, gt, rtol=1e-10, atol=1e-12)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    p = S.init_params(4)[0].astype(np.float64)
    X = rng.normal(0, 1, (33, 4))
    T = rng.normal(0, 1, (33, 2))
    _, g = mlp.loss_grad(p, X, T, round_bf16=False)
    idx = rng.choice(p.size, 60, replace=False)
    h = 1e-6
    for k in idx:
        q = p.copy(); q[k] += h; lp, _ = mlp.loss_grad(q, X, T, round_bf16=False)
        q[k] -= 2 * h; lm, _ = mlp.loss_grad(q, X, T, round_bf16=False)
        assert g[k] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)


def test_adam_matches_pytorch_optimizer():
    rng = np.random.default_rng(5)
    p = rng.normal(0, 1, 50)
    grads = rng.normal(0, 1, (4, 50))
    t = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    q = p.copy()
    for k in range(4):
        opt.zero_grad()
        t.grad = torch.tensor(grads[k])
        opt.step()
        q, m, v = mlp.adam(q, grads[k], m, v, k + 1, 1e-2)
    assert np.allclose(q, t.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_training_reduces_loss():
    rng = np.random.default_rng(6)
    X = rng.normal(0, 1, (256, 4))
    T = np.stack([np.sin(X[:, 0]) + 0.5 * X[:, 1], X[:, 2] * X[:, 3]], 1)
    p = S.init_params(7)[0].astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0, _ = mlp.loss_grad(p, X, T)
    for k in range(200):
        _, g = mlp.loss_grad(p, X, T)
        p, m, v = mlp.adam(p, g, m, v, k + 1, 3e-3)
    l1, _ = mlp.loss_grad(p, X, T)
    assert l1 < 0.3 * l0
