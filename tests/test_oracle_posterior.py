"""Pins for the posterior-draw oracle (oracle/posterior.py; Sec. 5,
Eq. thompson_sample): the posterior from another route (conditioning the
joint Gaussian through its precision matrix), the prior when there is no
data, interpolation of noise-free data, ARD against the isotropic kernel,
and the covariance of many draws."""
import numpy as np
import pytest

import ciq_inputs as ci
from oracle import ciq, kernels
from oracle import posterior as PO

LS = np.array([0.3, 0.5, 0.2])


def _data(n=40, nc=60, d=3, seed=3):
    Xtr = ci.points(seed, n, d)
    Xc = ci.points(seed + 1, nc, d)
    y = np.sin(6.0 * Xtr.sum(axis=1))
    return Xtr, y, Xc


@pytest.mark.parametrize("kind", ["rbf", "matern52"])
def test_posterior_equals_conditioning_through_the_joint_precision(kind):
    Xtr, y, Xc = _data()
    noise, s, m = 1e-2, 1.7, 0.3
    mu, cov = PO.posterior(Xtr, y, Xc, kind, LS, s, noise, 0.0, m)
    Xall = np.vstack([Xtr, Xc])
    S = PO.kernel_ard(Xall, Xall, kind, LS, s)
    S[:40, :40] += noise * np.eye(40)
    Lam = np.linalg.inv(S)
    cov2 = np.linalg.inv(Lam[40:, 40:])
    mu2 = m - cov2 @ Lam[40:, :40] @ (y - m)
    np.testing.assert_allclose(cov, cov2, rtol=0, atol=1e-8 * np.abs(cov2).max())
    np.testing.assert_allclose(mu, mu2, rtol=0, atol=1e-8 * np.abs(mu2).max())


def test_no_data_gives_the_prior_and_noise_free_data_are_interpolated():
    Xtr, y, Xc = _data()
    mu, cov = PO.posterior(np.zeros((0, 3)), np.zeros(0), Xc, "matern52", LS, 1.0, 1e-2, 1e-4, 0.5)
    np.testing.assert_allclose(cov, PO.kernel_ard(Xc, Xc, "matern52", LS, 1.0) + 1e-4 * np.eye(60), atol=1e-15)
    assert np.all(mu == 0.5)
    # Candidates that are training points, nearly noise-free data: mean = y, variance ~ jitter.
    Xc2 = np.vstack([Xtr[:10], Xc])
    mu, cov = PO.posterior(Xtr, y, Xc2, "matern52", LS, 1.0, 1e-10, 1e-4, 0.0)
    np.testing.assert_allclose(mu[:10], y[:10], atol=1e-6)
    np.testing.assert_allclose(np.diag(cov)[:10], 1e-4, atol=1e-6)
    assert np.linalg.eigvalsh(cov).min() > 1e-4 - 1e-9


def test_ard_with_equal_lengthscales_is_the_isotropic_kernel():
    X = ci.points(5, 30, 4)
    K1 = PO.kernel_ard(X, X, "matern52", np.full(4, 0.37), 1.3)
    K2 = kernels.kernel_matrix(X, X, "matern52", 0.37, 1.3)
    np.testing.assert_allclose(K1, K2, rtol=1e-14, atol=1e-15)


def test_draws_have_the_posterior_mean_and_covariance():
    Xtr, y, Xc = _data(n=15, nc=12)
    mu, cov = PO.posterior(Xtr, y, Xc, "rbf", LS, 1.0, 1e-3, 1e-4, 0.1)
    M = 40000
    eps = np.random.default_rng(0).standard_normal((M, 12))
    F = PO.thompson_draws(mu, cov, eps)
    np.testing.assert_allclose(F.mean(axis=0), mu, atol=5 * np.sqrt(np.diag(cov).max() / M))
    C = np.cov(F.T)
    assert np.abs(C - cov).max() < 6 * np.sqrt(2.0 / M) * np.diag(cov).max()


def test_ciq_on_the_posterior_covariance_converges_to_the_exact_draw():
    Xtr, y, Xc = _data(n=30, nc=200)
    mu, cov = PO.posterior(Xtr, y, Xc, "matern52", LS, 1.0, 1e-3, 1e-4, 0.0)
    eps = ci.rhs(8, 200, 3)
    exact = PO.thompson_draws(mu, cov, eps)
    lam = np.linalg.eigvalsh(cov)
    A, info = ciq.ciq_apply(ciq.dense_mvm(cov), eps, 16, "sqrt", tol=1e-10, max_iter=600, stop_rule="errbound",
                            lmin=1e-4, lmax=1.05 * lam[-1])
    got = mu[None, :] + A
    err = np.linalg.norm(got - exact, axis=1) / np.linalg.norm(exact - mu[None, :], axis=1)
    assert err.max() < 1e-6


def test_preconditioned_draws_use_a_root_of_the_posterior_covariance():
    # R R^T = COV* for the rotated root of the preconditioned draw (the draws'
    # covariance), checked on all N* columns of the identity; the rotation
    # differs from the principal root (R is not symmetric); eps = 0 gives the mean.
    Xtr, y, Xc = _data()
    jitter = 1e-3
    mu, cov = PO.posterior(Xtr, y, Xc, "matern52", LS, 1.2, 1e-2, jitter, 0.1)
    n = len(mu)
    D = PO.preconditioned_draws(mu, cov, jitter, 12, np.eye(n)) - mu[None, :]
    R = D.T                                                    # column c = R e_c
    assert np.abs(R @ R.T - cov).max() < 1e-10 * np.abs(cov).max()
    assert np.abs(R - R.T).max() > 1e-3 * np.abs(R).max()
    assert np.array_equal(PO.preconditioned_draws(mu, cov, jitter, 12, np.zeros((1, n)))[0], mu)


def test_full_rank_preconditioned_draws_are_the_principal_root_draws():
    # At full rank the pivoted Cholesky factor reproduces COV* - jitter I, so
    # P = COV*, A = P^{-1/2} COV* P^{-1/2} = I and R = P^{1/2} = COV*^{1/2}:
    # the preconditioned draw is the principal-root draw (O1).
    Xtr, y, Xc = _data()
    jitter = 1e-2
    mu, cov = PO.posterior(Xtr, y, Xc, "rbf", LS, 0.8, 1e-2, jitter, -0.3)
    n = len(mu)
    eps = ci.rhs(7, n, 3)
    got = PO.preconditioned_draws(mu, cov, jitter, n, eps)
    want = PO.thompson_draws(mu, cov, eps)
    assert np.abs(got - want).max() < 1e-8 * np.abs(want).max()
