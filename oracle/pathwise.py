"""Pathwise-conditioned posterior samples with a random-feature prior (oracle, FP64).

Test infrastructure only (see the package docstring).

Sec. 2.1 (eq. pathwise_conditoning): a sample of the GP posterior at test
points X* is

    f_n(X*) = f(X*) + k(X*, X) (K + lambda I)^{-1} (y - f(X) - zeta),
    zeta ~ N(0, lambda I),   f ~ GP(0, k),

with the solve done by an iterative method (ADASAP here).  The paper draws f
with q random features (2048 in its experiments, App. D.3) and takes 64 samples
for the test NLL (Sec. 5.1).

Readings (the paper does not spell these out):

  cross-covariance   the display writes k_n(X*, X) in front of the solve; the
      pathwise update of the works it cites uses the prior k(X*, X), which is
      also the only computable choice (k_n is the posterior the samples are
      meant to represent).  We take k(X*, X).
  random features    Rahimi & Recht (2007): for a stationary kernel with
      k(0) = sigma2 and spectral density p,
          f(x) = sqrt(2 sigma2 / q) * sum_l theta_l cos(omega_l . x + phase_l),
          theta_l ~ N(0, 1), phase_l ~ U[0, 2 pi), omega_l ~ p,
      so that E[f(x) f(x')] = k(x - x').  The spectral draws are built from
      independent inputs:
          RBF          omega_l = z_l / ell,                       z_l ~ N(0, I_d)
          Matern-nu    omega_l = z_l * sqrt(2 nu / u_l) / ell,    u_l ~ chi^2(2 nu)
      (the Matern-nu spectral density is a multivariate Student t with 2 nu
      degrees of freedom, scaled by 1 / ell; nu = 3/2 or 5/2).
  test NLL           mean over test points of -log N(y*; mu, var) with mu the
      posterior mean m_n(x*) and var the sample variance of the s samples at x*
      (divisor s - 1) plus the noise variance lambda.

Every random number (z, u, phase, theta, zeta) is an input, so the CUDA path
and this module consume the same draws.

Functions
---------
rf_frequencies(z, u, kernel, ell)           omega (q x d)
rf_prior(Xq, z, u, phase, theta, kernel, ell, sigma2)   f(Xq) (m x s)
pathwise_rhs(y, FX, zeta)                   y 1^T - f(X) - zeta  (n x s)
pathwise_samples(Xtest, X, W, Fstar, ...)   f(X*) + k(X*, X) W
pathwise_exact(...)                         the samples with a dense Cholesky solve
posterior_cov(Xtest, X, ...)                k(X*, X*) - k(X*, X) K_lambda^{-1} k(X, X*)
rmse_nll(mean, samples, ytest, noise)       (RMSE, mean NLL)
"""

import numpy as np

from . import gp
from . import kernels as K

NU = {K.MATERN32: 1.5, K.MATERN52: 2.5}


def rf_frequencies(z, u, kernel, ell):
    """Spectral frequencies omega_l (rows) of the kernel's random features."""
    z = np.asarray(z, dtype=np.float64)
    if kernel == K.RBF:
        return z / ell
    nu = NU[kernel]
    u = np.asarray(u, dtype=np.float64)
    return z * np.sqrt(2.0 * nu / u)[:, None] / ell


def rf_features(Xq, omega, phase, sigma2):
    """phi(x)_l = sqrt(2 sigma2 / q) cos(omega_l . x + phase_l), one row per point."""
    Xq = np.asarray(Xq, dtype=np.float64)
    q = omega.shape[0]
    return np.sqrt(2.0 * sigma2 / q) * np.cos(Xq @ omega.T + np.asarray(phase, dtype=np.float64)[None, :])


def rf_prior(Xq, z, u, phase, theta, kernel, ell, sigma2):
    """f(Xq) = phi(Xq) theta: s prior draws (columns of theta) at the points Xq."""
    omega = rf_frequencies(z, u, kernel, ell)
    return rf_features(Xq, omega, phase, sigma2) @ np.asarray(theta, dtype=np.float64)


def pathwise_rhs(y, FX, zeta):
    """Right-hand sides of the pathwise solve: column j is y - f_j(X) - zeta_j."""
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    return y[:, None] - np.asarray(FX, dtype=np.float64) - np.asarray(zeta, dtype=np.float64)


def pathwise_samples(Xtest, X, W, Fstar, kernel, ell, sigma2):
    """f(X*) + k(X*, X) W, with W = (K + lambda I)^{-1} (y - f(X) - zeta)."""
    return np.asarray(Fstar, dtype=np.float64) + K.kernel_apply(Xtest, X, W, kernel, ell, sigma2)


def pathwise_exact(Xtest, X, y, FX, Fstar, zeta, kernel, ell, sigma2, lam):
    """The samples of eq. pathwise_conditoning with the solve done by Cholesky."""
    W = gp.solve_dense(X, pathwise_rhs(y, FX, zeta), kernel, ell, sigma2, lam)
    return pathwise_samples(Xtest, X, W, Fstar, kernel, ell, sigma2)


def posterior_cov(Xtest, X, kernel, ell, sigma2, lam):
    """k_n(X*, X*) of Sec. 2, eq. post_eqns (the textbook posterior covariance)."""
    Kss = K.kernel_matrix(Xtest, Xtest, kernel, ell, sigma2)
    Ksx = K.kernel_matrix(Xtest, X, kernel, ell, sigma2)
    A = gp.solve_dense(X, Ksx.T, kernel, ell, sigma2, lam)
    return Kss - Ksx @ A


def rmse_nll(mean, samples, ytest, noise):
    """(RMSE of the posterior mean, mean NLL under N(mean, var_samples + noise))."""
    mean = np.asarray(mean, dtype=np.float64).reshape(-1)
    S = np.asarray(samples, dtype=np.float64)
    yt = np.asarray(ytest, dtype=np.float64).reshape(-1)
    err = yt - mean
    rmse = float(np.sqrt(np.mean(err * err)))
    var = S.var(axis=1, ddof=1) + noise
    nll = float(np.mean(0.5 * np.log(2.0 * np.pi * var) + err * err / (2.0 * var)))
    return rmse, nll
