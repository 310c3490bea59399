"""Pins for the oracle of the learned bound predictor (oracle/mlp.py): each
check ties it to something other than itself -- central finite differences,
hand-evaluated scalar loops, Adam's closed form, NumPy's moments."""
import numpy as np
import pytest

import ciq_inputs as ci
from oracle import mlp


def random_theta(seed):
    F = ci.normal(seed, 40 * mlp.N_IN).reshape(40, mlp.N_IN) * 3.0 + 1.0
    Y = ci.normal(seed + 1, 40 * mlp.N_OUT).reshape(40, mlp.N_OUT) * 2.0 - 1.0
    theta = mlp.init_params(seed + 2, mlp.normaliser(F, Y))
    # non-zero biases so every term of the chain rule is exercised
    theta[mlp.OFF_B1:mlp.OFF_W2] = 0.3 * ci.normal(seed + 3, mlp.N_HID)
    theta[mlp.OFF_B2:mlp.OFF_W3] = 0.3 * ci.normal(seed + 4, mlp.N_HID)
    theta[mlp.OFF_B3:] = 0.3 * ci.normal(seed + 5, mlp.N_OUT)
    return theta, F, Y


def test_layout_sizes():
    assert mlp.N_PARAMS == 82 + 38 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3 == 6933


def test_gradient_matches_central_differences():
    theta, F, Y = random_theta(11)
    _, g = mlp.loss_and_grad(theta, F[:7], Y[:7])
    rng_idx = list(range(mlp.OFF_W1, mlp.OFF_W1 + 5)) + list(range(mlp.OFF_B1, mlp.OFF_B1 + 3)) + \
        [mlp.OFF_W2 + 17, mlp.OFF_W2 + 64 * 9 + 40, mlp.OFF_B2 + 7, mlp.OFF_W3 + 5, mlp.OFF_W3 + 190,
         mlp.OFF_B3, mlp.OFF_B3 + 2, mlp.OFF_W1 + 37 * 64 + 63]
    h = 1e-6
    for k in rng_idx:
        tp = theta.copy()
        tm = theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (mlp.loss_and_grad(tp, F[:7], Y[:7])[0] - mlp.loss_and_grad(tm, F[:7], Y[:7])[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)), k
    # normaliser entries are not trained
    assert np.all(g[:mlp.OFF_W1] == 0)


def test_forward_matches_scalar_loops():
    theta, F, _ = random_theta(12)
    fmu, fsd, ymu, ysd, W1, b1, W2, b2, W3, b3 = mlp.unpack(theta)
    f = F[3]
    z = [(f[i] - fmu[i]) / fsd[i] for i in range(mlp.N_IN)]
    h1 = [np.tanh(b1[h] + sum(z[i] * W1[i, h] for i in range(mlp.N_IN))) for h in range(mlp.N_HID)]
    h2 = [np.tanh(b2[h] + sum(h1[k] * W2[k, h] for k in range(mlp.N_HID))) for h in range(mlp.N_HID)]
    y = [(b3[o] + sum(h2[h] * W3[h, o] for h in range(mlp.N_HID))) * ysd[o] + ymu[o] for o in range(mlp.N_OUT)]
    np.testing.assert_allclose(mlp.forward(theta, F[3:4])[4][0], y, rtol=1e-12)


def test_zero_first_layer_gives_constant_output():
    theta, F, _ = random_theta(13)
    theta[mlp.OFF_W1:mlp.OFF_B1] = 0.0
    Yh = mlp.forward(theta, F)[4]
    assert np.allclose(Yh, Yh[0], rtol=0, atol=1e-12)


def test_adam_first_steps_closed_form():
    # Constant gradient g: bias-corrected moments are g and g^2 at every
    # step, so each update is -lr g / (|g| + eps).
    theta = np.zeros(mlp.N_PARAMS)
    m = np.zeros(mlp.N_PARAMS)
    v = np.zeros(mlp.N_PARAMS)
    g = np.zeros(mlp.N_PARAMS)
    g[mlp.OFF_W1:] = np.linspace(-2.0, 3.0, mlp.N_PARAMS - mlp.OFF_W1)
    for step in range(1, 4):
        before = theta.copy()
        mlp.adam_step(theta, g, m, v, step, 0.01)
        delta = theta - before
        np.testing.assert_allclose(delta[mlp.OFF_W1:], -0.01 * g[mlp.OFF_W1:] / (np.abs(g[mlp.OFF_W1:]) + 1e-8),
                                   rtol=1e-9, atol=1e-15)
        assert np.all(delta[:mlp.OFF_W1] == 0)


def test_features_are_population_moments():
    X = np.array([[0.0, 1.0, 5.0], [2.0, 3.0, 5.0], [4.0, 2.0, 5.0], [2.0, 2.0, 5.0]])
    f = mlp.features(X, "matern52", 0.5, 2.0, 1e-3)
    assert f[0] == pytest.approx(np.log(4)) and f[1] == 3 and f[2] == 1.0
    assert f[3] == pytest.approx(np.log(0.5)) and f[4] == pytest.approx(np.log(2.0))
    assert f[5] == pytest.approx(np.log(1e-3))
    np.testing.assert_allclose(f[6:9], [2.0, 2.0, 5.0])
    np.testing.assert_allclose(f[22:25], [2.0, 0.5, 0.0])
    assert np.all(f[9:22] == 0) and np.all(f[25:] == 0)
    assert mlp.features(X, "rbf", 1.0, 1.0, 0.0)[5] == pytest.approx(np.log(1e-12))


def test_normaliser_standardises_columns():
    _, F, Y = random_theta(14)
    F[:, 5] = 7.0                      # a constant column keeps standard deviation 1
    norm = mlp.normaliser(F, Y)
    theta = np.zeros(mlp.N_PARAMS)
    theta[:mlp.OFF_W1] = norm
    Z0 = mlp.forward(theta, F)[0]
    np.testing.assert_allclose(Z0.mean(axis=0), 0.0, atol=1e-12)
    sd = Z0.std(axis=0)
    np.testing.assert_allclose(np.delete(sd, 5), 1.0, rtol=1e-12)
    assert norm[mlp.N_IN + 5] == 1.0


def test_minibatch_indices_follow_the_generator():
    idx = mlp.minibatch(99, 3, 16, 1000)
    u = ci.uniform(99, 48)[32:]
    assert np.array_equal(idx, np.floor(u * 1000).astype(np.int64))
    assert idx.min() >= 0 and idx.max() < 1000


def test_training_fits_a_smooth_function():
    n = 2000
    F = ci.uniform(21, n * mlp.N_IN).reshape(n, mlp.N_IN) * 2.0 - 1.0
    Y = np.stack([np.sin(2 * F[:, 0]) + F[:, 1] ** 2, F[:, 2] * F[:, 3] + 0.5 * F[:, 4],
                  np.cos(F[:, 0] - F[:, 5])], axis=1)
    theta = mlp.init_params(5, mlp.normaliser(F, Y))
    loss0 = mlp.loss_and_grad(theta, F, Y)[0]
    theta, _, _, losses = mlp.train(theta, F, Y, steps=1500, batch=64, lr=3e-3, seed=8)
    loss1 = mlp.loss_and_grad(theta, F, Y)[0]
    assert loss1 < 0.1 * loss0

