"""Pins of the FP64 reference network (CPU): central differences of the
loss, the all-zero network reducing to the Taylor weights, and Adam's first
step under a constant gradient."""
import numpy as np
import pytest

import oracle
from oracle import mlp


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.uniform(1.5, 4.5, n)
    X = mlp.features(v, 20.0, 1.6, 12.0)
    T = rng.standard_normal((n, 4))
    y = rng.standard_normal(n)
    w = rng.uniform(0.5, 2.0, n)
    return np.concatenate([X, T, y[:, None], w[:, None]], axis=1)


def test_parameter_count_and_packing():
    assert mlp.NPARAM == 64 * 4 + 64 + 64 * 64 + 64 + 8 * 64 + 8
    th = np.arange(mlp.NPARAM, dtype=np.float64)
    np.testing.assert_array_equal(mlp.pack(mlp.unpack(th)), th)


def test_zero_output_layer_gives_taylor_weights():
    c = oracle.fd_coefficients(4)
    th = mlp.init_params(0, scale_out=0.0)
    X = mlp.features(np.linspace(1.5, 4.5, 7), 20.0, 1.6, 12.0)
    np.testing.assert_allclose(mlp.coefficients(th, X, c), np.tile(c[1:], (7, 1)), rtol=0,
                               atol=0)


def test_loss_vanishes_when_targets_come_from_the_predicted_weights():
    c = oracle.fd_coefficients(4)
    th = mlp.init_params(1, scale_out=0.5)
    S = _samples(50, 2)
    S[:, 8] = np.sum(mlp.coefficients(th, S[:, :4], c) * S[:, 4:8], axis=1)
    assert mlp.loss(th, S, c) < 1e-28


@pytest.mark.parametrize("seed", [3, 4])
def test_loss_gradient_matches_central_differences(seed):
    c = oracle.fd_coefficients(4)
    th = mlp.init_params(seed, scale_out=0.7)
    S = _samples(40, seed + 10)
    L, g = mlp.loss_grad(th, S, c)
    assert abs(L - mlp.loss(th, S, c)) < 1e-14 * abs(L)
    rng = np.random.default_rng(seed)
    idx = np.concatenate([rng.choice(mlp.NPARAM, 200, replace=False),
                          np.arange(mlp.NPARAM - 8, mlp.NPARAM)])
    eps = 1e-6
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (mlp.loss(tp, S, c) - mlp.loss(tm, S, c)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-8, np.abs(g).max()), (i, fd, g[i])


def test_adam_first_step_is_lr_times_sign():
    th = np.linspace(-1, 1, 11)
    g = np.linspace(-3, 2, 11) + 0.05
    new, m, v = mlp.adam(th, g, np.zeros(11), np.zeros(11), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(new - th, -0.01 * np.sign(g), rtol=1e-12)


def _table_case():
    cT = oracle.fd_coefficients(4)
    th = mlp.init_params(3, scale_out=1.0)
    lo, hi, h, dt, f = 0.1, 0.45, 20.0, 1.6, 12.0
    C = np.random.default_rng(0).uniform(lo, hi, 4000)
    X = np.stack([C, np.full_like(C, h / 10), np.full_like(C, dt), np.full_like(C, f / 10)], 1)
    return cT, th, lo, hi, h, dt, f, C, mlp.coefficients(th, X, cT)


def test_table_weights_equal_the_network_at_the_nodes():
    cT, th, lo, hi, h, dt, f, _, _ = _table_case()
    n = 33
    Ci = np.sqrt(lo * lo + (hi * hi - lo * lo) * np.arange(n) / (n - 1))
    X = np.stack([Ci, np.full(n, h / 10), np.full(n, dt), np.full(n, f / 10)], 1)
    np.testing.assert_allclose(mlp.table_coefficients(th, Ci, h, dt, f, n, lo, hi, cT),
                               mlp.coefficients(th, X, cT), rtol=1e-13, atol=0)


def test_table_of_a_zero_network_is_the_taylor_stencil_everywhere():
    cT, _, lo, hi, h, dt, f, C, _ = _table_case()
    th0 = np.zeros(mlp.NPARAM)
    t = mlp.table_coefficients(th0, C, h, dt, f, 17, lo, hi, cT)
    np.testing.assert_array_equal(t, np.broadcast_to(cT[1:5], t.shape))


def test_table_clamps_outside_the_node_range_and_handles_one_velocity():
    cT, th, lo, hi, h, dt, f, _, _ = _table_case()
    t = mlp.table_coefficients(th, np.array([lo - 0.05, lo, hi, hi + 0.05]), h, dt, f, 9,
                               lo, hi, cT)
    np.testing.assert_array_equal(t[0], t[1])
    np.testing.assert_array_equal(t[2], t[3])
    same = mlp.table_coefficients(th, np.array([0.3, 0.3]), h, dt, f, 5, 0.3, 0.3, cT)
    X = np.array([[0.3, h / 10, dt, f / 10]])
    np.testing.assert_allclose(same, np.repeat(mlp.coefficients(th, X, cT), 2, 0), rtol=1e-13)


def test_table_weights_converge_to_the_network_at_second_order():
    """Linear interpolation error falls about 16x for 4x the nodes where the
    network is smooth (8x here, with the ReLU kinks); a slip in the
    interpolation weight (f against 1 - f) leaves first-order error (4x)."""
    cT, th, lo, hi, h, dt, f, C, direct = _table_case()

    def rms(n):
        t = mlp.table_coefficients(th, C, h, dt, f, n, lo, hi, cT)
        return np.sqrt(np.mean((t - direct) ** 2)) / np.sqrt(np.mean(direct ** 2))

    assert rms(32) / rms(128) > 6.0
    assert rms(256) < 1e-6
