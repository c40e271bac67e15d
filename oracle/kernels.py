"""Stationary covariance kernels and brute-force kernel products (oracle, FP64).

The paper uses RBF, Matern-3/2 and Matern-5/2 kernels (Table 1; Sec. 5.3 uses
Matern-3/2; the taxi run in Sec. 5.2 uses RBF) with a lengthscale and a kernel
variance (App. D.1), but never writes the formulas out.  We take the standard
forms, with r = ||x - x'||, lengthscale ell and variance sigma2:

    RBF         k(r) = sigma2 * exp(-r^2 / (2 ell^2))
    Matern-3/2  k(r) = sigma2 * (1 + a) * exp(-a),            a = sqrt(3) r / ell
    Matern-5/2  k(r) = sigma2 * (1 + a + a^2 / 3) * exp(-a),  a = sqrt(5) r / ell

and their derivatives with respect to ell (used by the hyperparameter adjoint):

    RBF         dk/dell = k * r^2 / ell^3
    Matern-3/2  dk/dell = sigma2 * a^2 * exp(-a) / ell
    Matern-5/2  dk/dell = sigma2 * a^2 * (1 + a) * exp(-a) / (3 ell)

dk/dsigma2 = k / sigma2 for all three.

Squared distances are formed in the difference form sum_k (x_k - y_k)^2, which
has no cancellation; this is the exact definition, not the fast expansion.
"""

import numpy as np

RBF = 0
MATERN32 = 1
MATERN52 = 2
NAMES = {RBF: "rbf", MATERN32: "matern32", MATERN52: "matern52"}

# elements per chunk in the brute-force products (keeps the m x n block small)
_CHUNK_ELEMS = 1 << 22


def sqdist(X1, X2):
    """Exact pairwise squared distances ||x_i - y_j||^2, difference form, FP64."""
    X1 = np.asarray(X1, dtype=np.float64)
    X2 = np.asarray(X2, dtype=np.float64)
    out = np.zeros((X1.shape[0], X2.shape[0]))
    for k in range(X1.shape[1]):
        diff = X1[:, k][:, None] - X2[:, k][None, :]
        out += diff * diff
    return out


def kernel_from_sqdist(r2, kernel, ell, sigma2):
    """k(r) for a matrix of squared distances r2 (standard forms above)."""
    r2 = np.maximum(np.asarray(r2, dtype=np.float64), 0.0)
    if kernel == RBF:
        return sigma2 * np.exp(-r2 / (2.0 * ell * ell))
    r = np.sqrt(r2)
    if kernel == MATERN32:
        a = np.sqrt(3.0) * r / ell
        return sigma2 * (1.0 + a) * np.exp(-a)
    if kernel == MATERN52:
        a = np.sqrt(5.0) * r / ell
        return sigma2 * (1.0 + a + a * a / 3.0) * np.exp(-a)
    raise ValueError("unknown kernel %r" % (kernel,))


def dkernel_dell_from_sqdist(r2, kernel, ell, sigma2):
    """dk/dell for a matrix of squared distances r2 (formulas above)."""
    r2 = np.maximum(np.asarray(r2, dtype=np.float64), 0.0)
    if kernel == RBF:
        return sigma2 * np.exp(-r2 / (2.0 * ell * ell)) * r2 / ell ** 3
    r = np.sqrt(r2)
    if kernel == MATERN32:
        a = np.sqrt(3.0) * r / ell
        return sigma2 * a * a * np.exp(-a) / ell
    if kernel == MATERN52:
        a = np.sqrt(5.0) * r / ell
        return sigma2 * a * a * (1.0 + a) * np.exp(-a) / (3.0 * ell)
    raise ValueError("unknown kernel %r" % (kernel,))


def kernel_matrix(X1, X2, kernel, ell, sigma2):
    """Dense K(X1, X2) (small problems only)."""
    return kernel_from_sqdist(sqdist(X1, X2), kernel, ell, sigma2)


def kernel_apply(Xr, Xc, W, kernel, ell, sigma2, deriv=False):
    """K(Xr, Xc) @ W by brute force in row chunks; never stores the full K.

    With deriv=True the kernel is replaced by dk/dell.  Xr: (m, d), Xc: (n, d),
    W: (n, s) or (n,).  Returns (m, s) (or (m,)).
    """
    Xr = np.asarray(Xr, dtype=np.float64)
    Xc = np.asarray(Xc, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    vec = W.ndim == 1
    W2 = W[:, None] if vec else W
    m, n = Xr.shape[0], Xc.shape[0]
    out = np.zeros((m, W2.shape[1]))
    step = max(1, _CHUNK_ELEMS // max(n, 1))
    f = dkernel_dell_from_sqdist if deriv else kernel_from_sqdist
    for i0 in range(0, m, step):
        Kc = f(sqdist(Xr[i0:i0 + step], Xc), kernel, ell, sigma2)
        out[i0:i0 + step] = Kc @ W2
    return out[:, 0] if vec else out


def kernel_rows(X, rows, W, kernel, ell, sigma2):
    """Block-row product K(X_B, X) @ W for row indices B (Alg. 2, Step I)."""
    X = np.asarray(X, dtype=np.float64)
    return kernel_apply(X[np.asarray(rows)], X, W, kernel, ell, sigma2)
