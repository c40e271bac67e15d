"""Pins for oracle.adasap and oracle.gp: dense linear algebra, special cases, convergence."""

import numpy as np
import pytest

from oracle import adasap as A
from oracle import gp
from oracle import kernels as K
from oracle import rng


def spd_lowrank(p, rank, rng_, decay=0.5, floor=1e-3):
    Q, _ = np.linalg.qr(rng_.standard_normal((p, p)))
    ev = np.concatenate([decay ** np.arange(rank) * 10.0, np.full(p - rank, floor)])
    return (Q * ev) @ Q.T


def test_nystrom_full_rank_reproduces_matrix():
    g = np.random.default_rng(0)
    M = spd_lowrank(24, 24, g, decay=0.8)
    Om = g.standard_normal((24, 24)) / np.sqrt(24)
    U, S, Delta = A.nystrom(M @ Om, Om, eps=0.0)
    np.testing.assert_allclose((U * S) @ U.T, M, atol=1e-9 * np.abs(M).max())
    U, S, Delta = A.nystrom(M @ Om, Om)                  # default shift: O(Delta) error
    assert Delta > 0
    np.testing.assert_allclose((U * S) @ U.T, M, atol=50 * Delta)


def test_nystrom_matches_pseudoinverse_definition():
    g = np.random.default_rng(1)
    M = spd_lowrank(40, 12, g)
    Om = g.standard_normal((40, 7)) / np.sqrt(40)
    Y = M @ Om
    ref = Y @ np.linalg.pinv(Om.T @ Y) @ Y.T            # Tropp et al. Nystrom definition
    U, S, _ = A.nystrom(Y, Om, eps=0.0)
    np.testing.assert_allclose((U * S) @ U.T, ref, atol=1e-10 * np.abs(ref).max())
    np.testing.assert_allclose(U.T @ U, np.eye(7), atol=1e-12)
    np.testing.assert_allclose(np.sort(S)[::-1], np.linalg.eigvalsh(ref)[::-1][:7], rtol=1e-9)


def test_nystrom_invariant_under_test_matrix_change_of_basis():
    g = np.random.default_rng(2)
    M = spd_lowrank(30, 10, g)
    Om = g.standard_normal((30, 6))
    Rm = g.standard_normal((6, 6)) + 3 * np.eye(6)
    U1, S1, _ = A.nystrom(M @ Om, Om, eps=0.0)
    U2, S2, _ = A.nystrom(M @ (Om @ Rm), Om @ Rm, eps=0.0)
    np.testing.assert_allclose((U1 * S1) @ U1.T, (U2 * S2) @ U2.T, atol=1e-9)


def test_nystrom_shift_and_clip():
    g = np.random.default_rng(3)
    Q, _ = np.linalg.qr(g.standard_normal((20, 3)))
    M = Q @ np.diag([5.0, 2.0, 1.0]) @ Q.T
    Om = g.standard_normal((20, 8)) / np.sqrt(20)
    U, S, Delta = A.nystrom(M @ Om, Om)
    assert np.all(S >= 0)
    np.testing.assert_allclose(S[:3], [5.0, 2.0, 1.0], rtol=1e-5)
    assert np.all(S[3:] < 10 * Delta)


def test_orthonormalize_is_the_positive_diagonal_thin_qr():
    g = np.random.default_rng(11)
    Om = g.standard_normal((40, 40)) / np.sqrt(40)          # square: badly conditioned
    Q = A.orthonormalize(Om)
    np.testing.assert_allclose(Q.T @ Q, np.eye(40), atol=1e-12)
    Rm = Q.T @ Om                                            # Om = Q R with R upper, diag > 0
    np.testing.assert_allclose(np.tril(Rm, -1), 0.0, atol=1e-12)
    assert np.all(np.diag(Rm) > 0)


def _random_nys(g, p=50, r=9, zeros=0):
    U, _ = np.linalg.qr(g.standard_normal((p, r)))
    S = np.sort(g.uniform(0.1, 10, r))[::-1]
    if zeros:
        S[-zeros:] = 0.0
    return U, S


@pytest.mark.parametrize("zeros", [0, 3])
def test_woodbury_inverse_forms_match_dense_solve(zeros):
    g = np.random.default_rng(4)
    U, S = _random_nys(g, zeros=zeros)
    rho = 0.37
    P = (U * S) @ U.T + rho * np.eye(50)
    G = g.standard_normal((50, 3))
    ref = np.linalg.solve(P, G)
    np.testing.assert_allclose(A.woodbury_inv_plain(U, S, rho, G), ref, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(A.woodbury_inv_stable(U, S, rho, G), ref, rtol=1e-10, atol=1e-12)
    v = g.standard_normal(50)
    lam, Q = np.linalg.eigh(P)
    ref_sqrt = Q @ ((Q.T @ v) / np.sqrt(lam))
    np.testing.assert_allclose(A.woodbury_inv_sqrt(U, S, rho, v), ref_sqrt, rtol=1e-10, atol=1e-12)


def test_stable_woodbury_survives_non_orthonormal_u():
    g = np.random.default_rng(5)
    U, S = _random_nys(g)
    U = U + 1e-3 * g.standard_normal(U.shape)
    rho = 0.2
    P = (U * S) @ U.T + rho * np.eye(50)
    x = g.standard_normal(50)
    np.testing.assert_allclose(A.woodbury_inv_stable(U, S, rho, x), np.linalg.solve(P, x), rtol=1e-9)
    assert np.linalg.norm(A.woodbury_inv_plain(U, S, rho, x) - np.linalg.solve(P, x)) > 1e-6


def test_get_stepsize_converges_to_top_preconditioned_eigenvalue():
    g = np.random.default_rng(6)
    p = 60
    H = spd_lowrank(p, 30, g, decay=0.85, floor=0.05)
    U, S = _random_nys(g, p=p, r=10)
    rho = 0.3
    P = (U * S) @ U.T + rho * np.eye(p)
    lam, Q = np.linalg.eigh(P)
    Pis = (Q / np.sqrt(lam)) @ Q.T
    top = np.linalg.eigvalsh(Pis @ H @ Pis)[-1]
    eta, lam_hat = A.get_stepsize(lambda v: H @ v, lambda v: A.woodbury_inv_sqrt(U, S, rho, v),
                                  g.standard_normal(p), N=400)
    assert abs(lam_hat - top) < 1e-9 * top
    assert abs(eta - 1 / top) < 1e-9 / top
    _, lam10 = A.get_stepsize(lambda v: H @ v, lambda v: A.woodbury_inv_sqrt(U, S, rho, v),
                              g.standard_normal(p), N=10)
    assert lam10 <= top * (1 + 1e-12) and lam10 > 0.5 * top


def _small_problem(n=240, d=3, seed=7, lam=0.1, kernel=K.RBF, ell=1.0):
    g = np.random.default_rng(seed)
    X = g.standard_normal((n, d))
    y = np.sin(X @ np.ones(d)) + 0.1 * g.standard_normal(n)
    return X, y[:, None], kernel, ell, 1.0, lam


def test_accel_params_hand_values_where_each_root_and_nu_matter():
    """Alg. 2's initialisation: beta = 1 - sqrt(mu/nu), gamma = 1/sqrt(mu nu),
    alpha = 1/(1 + gamma nu), against values worked out by hand.

    At (mu, nu) = (1/4, 16): mu/nu = 1/64 and mu nu = 4, so beta = 7/8,
    gamma = 1/2 and alpha = 1/9.  A dropped root gives beta = 63/64 or
    gamma = 1/4; a dropped nu in alpha gives 2/3; mu and nu swapped give
    beta = -7.  At (1/100, 4): beta = 1 - 1/20, gamma = 5, alpha = 1/21
    (gamma > 1 here, so gamma and 1/gamma are told apart as well)."""
    for (mu, nu), want in (((0.25, 16.0), (7 / 8, 1 / 2, 1 / 9)),
                           ((0.01, 4.0), (19 / 20, 5.0, 1 / 21))):
        got = A.accel_params(mu, nu)
        np.testing.assert_allclose(got, want, rtol=1e-15, atol=0)
    # the plausible slips all land elsewhere at the first point
    beta, gamma, alpha = A.accel_params(0.25, 16.0)
    for wrong in (1 - 0.25 / 16, 1 - np.sqrt(16 / 0.25)):
        assert abs(beta - wrong) > 0.1
    for wrong in (1 / (0.25 * 16), np.sqrt(0.25 * 16)):
        assert abs(gamma - wrong) > 0.2
    for wrong in (1 / (1 + gamma), 1 / (1 + 1 / (0.25 * 16) * 16), gamma * 16 / (1 + gamma * 16)):
        assert abs(alpha - wrong) > 0.05


def test_accel_params_special_case_mu_equals_nu_is_plain_sap():
    X, Y, kern, ell, s2, lam = _small_problem()
    beta, gamma, alpha = A.accel_params(1.0, 1.0)
    assert (beta, gamma, alpha) == (0.0, 1.0, 0.5)
    n, b, r = X.shape[0], 40, 12
    sched = rng.philox_schedule(n, b, r, seed=1)
    rec = []
    W3 = A.adasap(X, Y, kern, ell, s2, lam, b, r, 3, sched, mu=1.0, nu=1.0, record=rec)
    W = np.zeros_like(Y)
    for t in range(3):
        B, Om, v0 = sched(t)
        R = K.kernel_rows(X, B, W, kern, ell, s2) + lam * W[B] - Y[B]
        assert np.allclose(R, rec[t]["R"], atol=1e-13)
        W = W.copy()
        W[B] -= rec[t]["eta"] * rec[t]["D_B"]
    np.testing.assert_allclose(W3, W, atol=1e-13)
    W3lit = A.adasap(X, Y, kern, ell, s2, lam, b, r, 3, sched, mu=1.0, nu=1.0, nesterov="literal")
    assert np.abs(W3lit - W3).max() > 1e-6


def test_sap_exact_block_b_equals_n_is_one_step_solve():
    X, Y, kern, ell, s2, lam = _small_problem(n=150)
    Wstar = gp.solve_dense(X, Y, kern, ell, s2, lam)
    W1 = A.sap(X, Y, kern, ell, s2, lam, 150, 1, lambda t: np.arange(150))
    np.testing.assert_allclose(W1, Wstar, rtol=1e-10, atol=1e-10)


def test_sap_converges_and_tail_average_is_mean_of_last_half():
    X, Y, kern, ell, s2, lam = _small_problem(n=120)
    blocks = lambda t: rng.sample_block(120, 30, seed=2, t=t)
    Wstar = gp.solve_dense(X, Y, kern, ell, s2, lam)
    W = A.sap(X, Y, kern, ell, s2, lam, 30, 400, blocks)
    assert np.linalg.norm(W - Wstar) / np.linalg.norm(Wstar) < 1e-6
    T = 7
    hist = [A.sap(X, Y, kern, ell, s2, lam, 30, t, blocks) for t in range(T + 1)]
    Wbar = A.sap(X, Y, kern, ell, s2, lam, 30, T, blocks, tail_average=True)
    np.testing.assert_allclose(Wbar, np.mean(hist[4:], axis=0), atol=1e-14)


@pytest.mark.parametrize("variant", [("z", "standard"), ("w", "literal")])
@pytest.mark.parametrize("kernel", [K.RBF, K.MATERN32, K.MATERN52])
def test_adasap_converges_to_cholesky_solution(variant, kernel):
    X, Y, kern, ell, s2, lam = _small_problem(n=300, kernel=kernel, lam=0.3)
    n, b, r = 300, 100, 40
    Wstar = gp.solve_dense(X, Y, kern, ell, s2, lam)
    sched = rng.philox_schedule(n, b, r, seed=4)
    W = A.adasap(X, Y, kern, ell, s2, lam, b, r, 150, sched, point=variant[0], nesterov=variant[1])
    assert np.linalg.norm(W - Wstar) / np.linalg.norm(Wstar) < 2e-4
    assert gp.rel_residual(X, W, Y, kern, ell, s2, lam) < 3e-5


def test_adasap_identity_preconditioner_converges():
    X, Y, kern, ell, s2, lam = _small_problem(n=200, lam=0.3)
    sched = rng.philox_schedule(200, 50, 10, seed=5)
    res = [gp.rel_residual(X, A.adasap(X, Y, kern, ell, s2, lam, 50, 10, T, sched,
                                       precond="identity"), Y, kern, ell, s2, lam)
           for T in (100, 300)]
    # ADASAP-I (P_B = I) converges, more slowly than ADASAP (Table 1)
    assert res[1] < 0.05 and res[1] < 0.5 * res[0]


def test_adasap_multi_rhs_equals_columnwise_solves():
    X, Y1, kern, ell, s2, lam = _small_problem(n=160)
    g = np.random.default_rng(9)
    Y = np.concatenate([Y1, g.standard_normal((160, 2))], axis=1)
    sched = rng.philox_schedule(160, 40, 8, seed=6)
    Wm = A.adasap(X, Y, kern, ell, s2, lam, 40, 8, 20, sched)
    for c in range(3):
        Wc = A.adasap(X, Y[:, c], kern, ell, s2, lam, 40, 8, 20, sched)
        # the stepsize is shared across columns (one block, one preconditioner)
        np.testing.assert_allclose(Wm[:, c], Wc, atol=1e-12)


def test_residual_and_posterior_mean_definitions():
    X, Y, kern, ell, s2, lam = _small_problem(n=100)
    Wstar = gp.solve_dense(X, Y, kern, ell, s2, lam)
    assert gp.rel_residual(X, Wstar, Y, kern, ell, s2, lam) < 1e-12
    Km = K.kernel_matrix(X, X, kern, ell, s2)
    Wr = np.random.default_rng(1).standard_normal(Y.shape)
    full = np.linalg.norm(Km @ Wr + lam * Wr - Y) / np.linalg.norm(Y)
    assert abs(gp.rel_residual(X, Wr, Y, kern, ell, s2, lam) - full) < 1e-12
    assert abs(gp.rel_residual(X, Wr, Y, kern, ell, s2, lam, rows=np.arange(100)) - full) < 1e-12
    Xt = np.random.default_rng(2).standard_normal((13, 3))
    np.testing.assert_allclose(gp.posterior_mean(Xt, X, Wstar, kern, ell, s2),
                               K.kernel_matrix(Xt, X, kern, ell, s2) @ Wstar, atol=1e-12)
    W0 = gp.solve_dense(X[:40], Y[:40], kern, ell, s2, 1e-10)
    np.testing.assert_allclose(gp.posterior_mean(X[:40], X[:40], W0, kern, ell, s2), Y[:40], atol=1e-5)


@pytest.mark.parametrize("kernel", [K.RBF, K.MATERN32, K.MATERN52])
def test_hypergrad_by_finite_differences(kernel):
    X, Y, kern, ell, s2, lam = _small_problem(n=90, kernel=kernel, ell=0.8)
    g = np.random.default_rng(10)
    W = g.standard_normal((90, 2))
    G = g.standard_normal((90, 2))
    d_ell, d_s2 = gp.hypergrad(X, W, G, kern, ell, s2)
    f = lambda e, s: np.sum(G * K.kernel_apply(X, X, W, kern, e, s))
    h = 1e-6
    assert abs(d_ell - (f(ell + h, s2) - f(ell - h, s2)) / (2 * h)) < 1e-6 * (1 + abs(d_ell))
    assert abs(d_s2 - (f(ell, s2 + h) - f(ell, s2 - h)) / (2 * h)) < 1e-6 * (1 + abs(d_s2))


def test_hypergrad_gives_derivative_of_data_fit_term():
    X, Y, kern, ell, s2, lam = _small_problem(n=120, kernel=K.MATERN52, ell=0.9)

    def fit(e, s):
        return float(Y[:, 0] @ gp.solve_dense(X, Y, kern, e, s, lam)[:, 0])

    W = gp.solve_dense(X, Y, kern, ell, s2, lam)
    d_ell, d_s2 = gp.hypergrad(X, W, W, kern, ell, s2)
    h = 1e-6
    fd_ell = (fit(ell + h, s2) - fit(ell - h, s2)) / (2 * h)
    fd_s2 = (fit(ell, s2 + h) - fit(ell, s2 - h)) / (2 * h)
    assert abs(-d_ell - fd_ell) < 1e-5 * abs(fd_ell)
    assert abs(-d_s2 - fd_s2) < 1e-5 * abs(fd_s2)
