"""Surrogate network kernels against the FP64 oracle: forward, gradient and
Adam with the same bfloat16-rounded weights; training reduces the loss; the
ensemble spread is the members' sample deviation."""

import numpy as np
import pytest

from oracle import mlp
from workloads import surrogate as S
from gpu_common import B, normwise

pytestmark = pytest.mark.gpu


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = np.stack([10 ** rng.uniform(-2, 0, n), rng.uniform(0, 0.1, n), rng.uniform(0, 0.2, n),
                  rng.uniform(0.2, 2.0, n)], 1).astype(np.float32)
    Y = np.stack([X[:, 0] * (1 + 3 * X[:, 2]) + 0.1 * X[:, 3], np.sin(5 * X[:, 1]) + X[:, 3]], 1).astype(np.float32)
    return X, Y


def _standardize(X, Y):
    X = X.astype(np.float64)
    Y = Y.astype(np.float64)
    st = mlp.Standardizer(X, Y)
    return st, st.x(X), st.y(Y)


def test_loss_and_gradient_match_oracle():
    bd = B()
    M = 3
    P = S.init_params(11, M)
    X, Y = _data(1000, 1)             # not a multiple of the block size
    h = bd.tdpd_mlp_create(M)
    try:
        bd.tdpd_mlp_set_params(h, P)
        bd.tdpd_mlp_set_data(h, X, Y)
        loss, grad = bd.tdpd_mlp_loss_grad(h, M)
    finally:
        bd.tdpd_mlp_destroy(h)
    st, Xn, Yn = _standardize(X, Y)
    for k in range(M):
        lo, go = mlp.loss_grad(P[k], Xn.astype(np.float32).astype(np.float64),
                               Yn.astype(np.float32).astype(np.float64))
        assert loss[k] == pytest.approx(lo, rel=1e-5)
        assert normwise(grad[k], go) < 1e-5


def test_adam_steps_match_oracle():
    bd = B()
    P = S.init_params(12, 2)
    X, Y = _data(512, 2)
    h = bd.tdpd_mlp_create(2)
    try:
        bd.tdpd_mlp_set_params(h, P)
        bd.tdpd_mlp_set_data(h, X, Y)
        bd.tdpd_mlp_train(h, 3, 1e-3, 2)
        Pg = bd.tdpd_mlp_get_params(h, 2)
    finally:
        bd.tdpd_mlp_destroy(h)
    _, Xn, Yn = _standardize(X, Y)
    Xn = Xn.astype(np.float32).astype(np.float64)
    Yn = Yn.astype(np.float32).astype(np.float64)
    for k in range(2):
        p = P[k].astype(np.float64)
        m = np.zeros_like(p)
        v = np.zeros_like(p)
        for t in range(3):
            _, g = mlp.loss_grad(p.astype(np.float32), Xn, Yn)
            p, m, v = mlp.adam(p, g, m, v, t + 1, 1e-3)
        step = p - P[k]
        assert normwise(Pg[k] - P[k], step) < 1e-3
        assert np.abs(Pg[k] - p).max() < 1e-5


def test_training_reduces_loss_and_spread_is_member_deviation():
    bd = B()
    M = 5
    X, Y = _data(2048, 3)
    h = bd.tdpd_mlp_create(M)
    try:
        bd.tdpd_mlp_set_params(h, S.init_params(13, M))
        bd.tdpd_mlp_set_data(h, X, Y)
        l0, _ = bd.tdpd_mlp_loss_grad(h, M)
        l1 = bd.tdpd_mlp_train(h, 1500, 3e-3, M)
        Xt, Yt = _data(256, 4)
        mean, spread, each = bd.tdpd_mlp_predict(h, Xt, M)
    finally:
        bd.tdpd_mlp_destroy(h)
    assert (l1 < 0.05 * l0).all(), (l0, l1)
    assert np.allclose(mean, each.mean(0), rtol=1e-5, atol=1e-6)
    sd = each.astype(np.float64).std(0, ddof=1)
    assert np.allclose(spread, sd / np.abs(each.astype(np.float64).mean(0)), rtol=1e-3, atol=1e-6)
    rel = np.abs(mean - Yt) / (np.abs(Yt) + 0.1)
    assert np.median(rel) < 0.05


def test_training_and_prediction_throughput():
    """Timing of the surrogate's kernels at the sweep's sizes (5 members,
    4096 training samples; 2048 candidates to rank): Adam steps per second
    and samples per second, and the multiply-adds per second against the
    FP32 FMA rate of 152 SMs x 128 lanes x 2 flops x the SM clock (reported;
    the matrices are too small to fill the GPU, so the kernels are bound by
    launch latency)."""
    import time
    bd = B()
    M, n = 5, 4096
    X, Y = _data(n, 21)
    h = bd.tdpd_mlp_create(M)
    bd.tdpd_mlp_set_params(h, S.init_params(3, M))
    bd.tdpd_mlp_set_data(h, X, Y)
    bd.tdpd_mlp_train(h, 20, 1e-3, M)                        # warm-up
    steps = 500
    t0 = time.perf_counter()
    bd.tdpd_mlp_train(h, steps, 1e-3, M)
    t_step = (time.perf_counter() - t0) / steps
    Xc, _ = _data(2048, 22)
    bd.tdpd_mlp_predict(h, Xc, M)
    reps = 200
    t0 = time.perf_counter()
    for _ in range(reps):
        bd.tdpd_mlp_predict(h, Xc, M)
    t_pred = (time.perf_counter() - t0) / reps
    bd.tdpd_mlp_destroy(h)
    macs = 4 * 64 + 64 * 64 + 64 * 2                          # per sample and member, forward
    flops_step = 2 * 3 * macs * n * M                         # forward + two backward products
    peak = 152 * 128 * 2 * 2.07e9
    print('mlp: Adam step %.1f us (%.0f samples/s, %.2f TFLOP/s = %.2f %% of FP32 FMA peak); '
          'predict 2048 x %d members %.1f us' % (t_step * 1e6, n / t_step, flops_step / t_step / 1e12,
                                                 100 * flops_step / t_step / peak, M, t_pred * 1e6))
    assert t_step < 2e-3 and t_pred < 5e-3
