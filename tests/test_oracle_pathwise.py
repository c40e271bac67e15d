"""Pins of oracle/pathwise.py (pathwise-conditioned posterior samples, Sec. 2.1).

Each pin checks the oracle against something other than itself: the kernel the
random features must reproduce in expectation (Monte Carlo with a stated
error bound), the textbook posterior mean and covariance of Sec. 2 (eq.
post_eqns) that the pathwise update must have as its law, and scipy's normal
log-density for the NLL.
"""

import numpy as np
import pytest
from scipy import stats

from oracle import gp
from oracle import kernels as K
from oracle import pathwise as PW


def _draws(rng, q, d, kernel, s=1):
    z = rng.standard_normal((q, d))
    u = rng.chisquare(2 * PW.NU[kernel], q) if kernel != K.RBF else None
    phase = rng.uniform(0.0, 2.0 * np.pi, q)
    theta = rng.standard_normal((q, s))
    return z, u, phase, theta


@pytest.mark.parametrize("kernel", [K.RBF, K.MATERN32, K.MATERN52])
def test_random_features_reproduce_the_kernel(kernel):
    """E[phi(x) . phi(x')] = k(x - x') (Rahimi & Recht).  Each entry of phi phi^T is a
    mean of q independent terms of size <= 2 sigma2 / q, so its standard deviation is
    at most 2 sigma2 / sqrt(q); the check allows 5 of them.  Points are spread over
    distances ~ ell, where the three kernels differ by 0.04 .. 0.12 sigma2."""
    rng = np.random.default_rng(kernel)
    q, d, ell, sigma2 = 1 << 19, 3, 0.7, 1.6
    X = rng.standard_normal((8, d)) * 0.6
    z, u, phase, _ = _draws(rng, q, d, kernel)
    Phi = PW.rf_features(X, PW.rf_frequencies(z, u, kernel, ell), phase, sigma2)
    Kref = K.kernel_matrix(X, X, kernel, ell, sigma2)
    assert np.abs(Phi @ Phi.T - Kref).max() < 5 * 2 * sigma2 / np.sqrt(q)
    # the same features scored against a different kernel fail the bound
    other = K.RBF if kernel != K.RBF else K.MATERN32
    assert np.abs(Phi @ Phi.T - K.kernel_matrix(X, X, other, ell, sigma2)).max() > 5 * 2 * sigma2 / np.sqrt(q)


def _pathwise_map(Xt, X, kernel, ell, sigma2, lam):
    """The pathwise update is linear in (f(X), f(X*), zeta) for y = 0: probe it with unit
    inputs to get its matrix M (m x (2n + m))."""
    n, m = X.shape[0], Xt.shape[0]
    cols = 2 * n + m
    FX = np.zeros((n, cols))
    FX[:, :n] = np.eye(n)
    Fs = np.zeros((m, cols))
    Fs[:, n:n + m] = np.eye(m)
    Z = np.zeros((n, cols))
    Z[:, n + m:] = np.eye(n)
    return PW.pathwise_exact(Xt, X, np.zeros(n), FX, Fs, Z, kernel, ell, sigma2, lam)


@pytest.mark.parametrize("kernel", [K.RBF, K.MATERN52])
def test_pathwise_update_has_the_posterior_law(kernel):
    """With f ~ GP(0, k) and zeta ~ N(0, lambda I), f(X*) + k(X*, X) K_lambda^{-1}(y - f(X) - zeta)
    is Gaussian with mean m_n(X*) and covariance k_n(X*, X*) (Sec. 2, eq. post_eqns)."""
    rng = np.random.default_rng(10 + kernel)
    n, m, d, ell, sigma2, lam = 20, 5, 2, 0.8, 1.3, 0.4
    X = rng.standard_normal((n, d))
    Xt = rng.standard_normal((m, d))
    y = rng.standard_normal(n)
    M = _pathwise_map(Xt, X, kernel, ell, sigma2, lam)
    Xall = np.vstack([X, Xt])
    C = np.zeros((2 * n + m, 2 * n + m))
    C[:n + m, :n + m] = K.kernel_matrix(Xall, Xall, kernel, ell, sigma2)
    C[n + m:, n + m:] = lam * np.eye(n)
    cov = M @ C @ M.T
    np.testing.assert_allclose(cov, PW.posterior_cov(Xt, X, kernel, ell, sigma2, lam), atol=1e-10)
    # the mean: the update with f = 0, zeta = 0 is the posterior mean
    zero_n, zero_m = np.zeros((n, 1)), np.zeros((m, 1))
    mean = PW.pathwise_exact(Xt, X, y, zero_n, zero_m, zero_n, kernel, ell, sigma2, lam)
    ref = gp.posterior_mean(Xt, X, gp.solve_dense(X, y[:, None], kernel, ell, sigma2, lam), kernel, ell, sigma2)
    np.testing.assert_allclose(mean, ref, atol=1e-12)
    # a dropped noise term is visible: the covariance without zeta differs from k_n
    C2 = C.copy()
    C2[n + m:, n + m:] = 0.0
    assert np.abs(M @ C2 @ M.T - cov).max() > 1e-3


def test_random_feature_samples_have_the_posterior_covariance():
    """rf_prior and the pathwise update together: the sample covariance of 4000 samples
    (4096 random features) is within Monte Carlo error of k_n(X*, X*)."""
    rng = np.random.default_rng(21)
    n, m, d, ell, sigma2, lam, q, S = 15, 4, 2, 0.9, 1.0, 0.3, 4096, 4000
    X = rng.standard_normal((n, d))
    Xt = rng.standard_normal((m, d))
    z, u, phase, theta = _draws(rng, q, d, K.MATERN32, s=S)
    FX = PW.rf_prior(X, z, u, phase, theta, K.MATERN32, ell, sigma2)
    Fs = PW.rf_prior(Xt, z, u, phase, theta, K.MATERN32, ell, sigma2)
    zeta = rng.standard_normal((n, S)) * np.sqrt(lam)
    samples = PW.pathwise_exact(Xt, X, np.zeros(n), FX, Fs, zeta, K.MATERN32, ell, sigma2, lam)
    cov_ref = PW.posterior_cov(Xt, X, K.MATERN32, ell, sigma2, lam)
    # sampling error ~ sqrt(2 / S) sigma2 = 0.022, random-feature error ~ 2 / sqrt(q) = 0.03
    assert np.abs(np.cov(samples) - cov_ref).max() < 0.15
    assert np.abs(samples.mean(axis=1)).max() < 5 * np.sqrt(np.diag(cov_ref).max() / S)


def test_rmse_and_nll_against_scipy():
    rng = np.random.default_rng(3)
    m, s, noise = 50, 64, 0.05
    mean = rng.standard_normal(m)
    samples = mean[:, None] + 0.3 * rng.standard_normal((m, s))
    yt = mean + 0.2 * rng.standard_normal(m)
    rmse, nll = PW.rmse_nll(mean, samples, yt, noise)
    var = np.var(samples, axis=1, ddof=1) + noise
    assert rmse == pytest.approx(np.sqrt(np.mean((yt - mean) ** 2)), rel=1e-14)
    assert nll == pytest.approx(-np.mean(stats.norm.logpdf(yt, loc=mean, scale=np.sqrt(var))), rel=1e-12)
    # identical samples: the variance is the noise alone
    _, nll0 = PW.rmse_nll(mean, np.repeat(mean[:, None], 4, axis=1), yt, noise)
    assert nll0 == pytest.approx(-np.mean(stats.norm.logpdf(yt, loc=mean, scale=np.sqrt(noise))), rel=1e-12)
