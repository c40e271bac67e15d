"""Dense GP references: exact solve, posterior mean, residuals, adjoint (oracle, FP64).

  solve_dense     W* = (K + lambda I)^{-1} Y by Cholesky -- the target every
                  iterative solver of the paper converges to (Sec. 2, eq. post_eqns).
  posterior_mean  m_n(X*) = k(X*, X) W with a zero prior mean (App. D.1 uses a
                  zero-mean prior).
  rel_residual    ||(K + lambda I) W - Y||_F / ||Y||_F, on all rows or on a
                  subset of rows (scaled by sqrt(n / |rows|)).
  hypergrad       d_ell    = sum_c G[:, c]^T (dK/dell) W[:, c]
                  d_sigma2 = sum_c G[:, c]^T (dK/dsigma2) W[:, c]
                  With W = (K + lambda I)^{-1} y and G = W this is the building
                  block of d(y^T W)/dtheta = -W^T (dK/dtheta) W used when the
                  kernel hyperparameters are fitted (App. D.1).
  subspace_rel_error  ||proj_l(m_hat) - proj_l(m_n)||_H^2 / ||proj_l(m_n)||_H^2, the
                  error of a posterior-mean estimate m_hat = k(., X) w along the top-l
                  spectral basis functions (Sec. 3, Thm. main; the tail-averaging
                  experiment of the appendix), via the identity
                  ||proj_l(m') - proj_l(m_n)||_H^2 = ||Q_l (w - w*)||_K^2 with Q_l the
                  projector onto the top-l eigenvectors of K (App. proof of the
                  main theorem).
"""

import numpy as np
import scipy.linalg as sla

from . import kernels as K


def solve_dense(X, Y, kernel, ell, sigma2, lam):
    Kl = K.kernel_matrix(X, X, kernel, ell, sigma2) + lam * np.eye(X.shape[0])
    return sla.cho_solve(sla.cho_factor(Kl, lower=True), np.asarray(Y, dtype=np.float64))


def posterior_mean(Xtest, X, W, kernel, ell, sigma2):
    return K.kernel_apply(Xtest, X, W, kernel, ell, sigma2)


def rel_residual(X, W, Y, kernel, ell, sigma2, lam, rows=None):
    X = np.asarray(X, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n = X.shape[0]
    if rows is None:
        rows = np.arange(n)
    rows = np.asarray(rows)
    Rb = K.kernel_apply(X[rows], X, W, kernel, ell, sigma2) + lam * W[rows] - Y[rows]
    num = np.sqrt(np.sum(Rb * Rb) * n / len(rows))
    return float(num / np.sqrt(np.sum(Y * Y)))


def hypergrad(X, W, G, kernel, ell, sigma2):
    """(d_ell, d_sigma2) = (sum G * (dK/dell) W, sum G * (K / sigma2) W)."""
    X = np.asarray(X, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    dKW = K.kernel_apply(X, X, W, kernel, ell, sigma2, deriv=True)
    KW = K.kernel_apply(X, X, W, kernel, ell, sigma2)
    return float(np.sum(G * dKW)), float(np.sum(G * KW) / sigma2)


def subspace_rel_error(evals, evecs, w, wstar, top):
    """||Q_l (w - w*)||_K^2 / ||Q_l w*||_K^2 for l = top.

    evals, evecs: the eigenpairs of K in descending order (evecs[:, i] the i-th);
    ||Q_l z||_K^2 = sum_{i <= l} lambda_i (v_i^T z)^2 because Q_l and K commute."""
    V = np.asarray(evecs, dtype=np.float64)[:, :top]
    lam = np.asarray(evals, dtype=np.float64)[:top]
    num = np.sum(lam * (V.T @ (np.asarray(w, np.float64) - np.asarray(wstar, np.float64))) ** 2)
    den = np.sum(lam * (V.T @ np.asarray(wstar, np.float64)) ** 2)
    return float(num / den)
