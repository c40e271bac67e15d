"""Pins for oracle.kernels: closed forms against independent library routines."""

import numpy as np
import pytest
from scipy import special, stats
from scipy.spatial.distance import cdist

from oracle import kernels as K


def matern_bessel(r, nu, ell, sigma2):
    """General Matern kernel through the modified Bessel function K_nu (scipy)."""
    r = np.asarray(r, dtype=np.float64)
    z = np.sqrt(2.0 * nu) * r / ell
    out = np.full_like(z, sigma2)
    nz = z > 0
    out[nz] = sigma2 * 2.0 ** (1.0 - nu) / special.gamma(nu) * z[nz] ** nu * special.kv(nu, z[nz])
    return out


@pytest.mark.parametrize("kernel,nu", [(K.MATERN32, 1.5), (K.MATERN52, 2.5)])
@pytest.mark.parametrize("ell,sigma2", [(0.3, 1.0), (1.7, 2.5)])
def test_matern_half_integer_forms_match_bessel(kernel, nu, ell, sigma2):
    r = np.concatenate([[0.0, 1e-6], np.linspace(0.01, 6.0, 400)])
    got = K.kernel_from_sqdist(r * r, kernel, ell, sigma2)
    ref = matern_bessel(r, nu, ell, sigma2)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("ell,sigma2", [(0.5, 1.0), (2.0, 0.7)])
def test_rbf_matches_gaussian_density(ell, sigma2):
    rng = np.random.default_rng(1)
    d = 5
    X = rng.standard_normal((30, d))
    Y = rng.standard_normal((20, d))
    got = K.kernel_matrix(X, Y, K.RBF, ell, sigma2)
    norm_const = (2.0 * np.pi * ell * ell) ** (d / 2.0)
    ref = np.array([[sigma2 * norm_const * stats.multivariate_normal.pdf(x, mean=y, cov=ell * ell)
                     for y in Y] for x in X])
    np.testing.assert_allclose(got, ref, rtol=1e-10)


def test_matern_tends_to_rbf_for_large_nu():
    # Matern-nu -> RBF as nu -> infinity; evaluate the Bessel form in log space
    r = np.linspace(0.01, 3.0, 50)
    nu = 60.0
    z = np.sqrt(2.0 * nu) * r
    big = np.exp((1.0 - nu) * np.log(2.0) - special.gammaln(nu) + nu * np.log(z)
                 + np.log(special.kve(nu, z)) - z)
    rbf = K.kernel_from_sqdist(r * r, K.RBF, 1.0, 1.0)
    np.testing.assert_allclose(rbf, big, atol=5e-3)


def test_sqdist_matches_scipy_cdist():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((37, 11)) * 3 + 5
    B = rng.standard_normal((29, 11)) * 3 + 5
    np.testing.assert_allclose(K.sqdist(A, B), cdist(A, B, "sqeuclidean"), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kernel", [K.RBF, K.MATERN32, K.MATERN52])
def test_lengthscale_derivative_by_finite_differences(kernel):
    r = np.linspace(0.0, 5.0, 101)
    ell, sigma2, h = 0.8, 1.3, 1e-5
    got = K.dkernel_dell_from_sqdist(r * r, kernel, ell, sigma2)
    fd = (K.kernel_from_sqdist(r * r, kernel, ell + h, sigma2)
          - K.kernel_from_sqdist(r * r, kernel, ell - h, sigma2)) / (2 * h)
    np.testing.assert_allclose(got, fd, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("kernel", [K.RBF, K.MATERN32, K.MATERN52])
def test_kernel_matrix_is_psd_with_constant_diagonal(kernel):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((120, 4))
    Km = K.kernel_matrix(X, X, kernel, 0.9, 2.0)
    np.testing.assert_allclose(np.diag(Km), 2.0, rtol=0, atol=0)
    assert np.linalg.eigvalsh(Km).min() > -1e-10


def test_kernel_apply_chunking_and_row_indexing(monkeypatch):
    rng = np.random.default_rng(4)
    X = rng.standard_normal((203, 6))
    W = rng.standard_normal((203, 3))
    rows = rng.choice(203, size=57, replace=False)
    dense = K.kernel_matrix(X[rows], X, K.MATERN52, 1.1, 0.8) @ W
    monkeypatch.setattr(K, "_CHUNK_ELEMS", 203 * 5 + 1)   # force many ragged chunks
    got = K.kernel_rows(X, rows, W, K.MATERN52, 1.1, 0.8)
    np.testing.assert_allclose(got, dense, rtol=1e-12, atol=1e-12)
    e = np.zeros(203)
    e[17] = 1.0
    col = K.kernel_rows(X, rows, e, K.MATERN52, 1.1, 0.8)
    np.testing.assert_allclose(col, K.kernel_matrix(X[rows], X[17:18], K.MATERN52, 1.1, 0.8)[:, 0])
