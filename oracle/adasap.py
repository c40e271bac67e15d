"""ADASAP and its sub-routines, restated step by step in FP64 (oracle).

Follows, in the paper's order and notation:
  Alg. 1  SAP for K_lambda W = Y (exact block solve; optional tail averaging)
  Alg. 2  ADASAP (Steps I-IV)
  Alg. 4  RandNysAppx (randomized Nystrom approximation)
  App. C.2  Woodbury applies: the plain inverse (eq. inv_nys_woodbury), the
            Cholesky-stabilised inverse, and the inverse square root
            (eq. inv_sqrt_nys_woodbury)
  Alg. 5  GetStepsize (randomized powering)
  Alg. 6  NesterovAcc

Readings of places where the paper is silent, garbled or inconsistent (each is
a keyword argument here so that tests can discriminate between them):

  point='z' (default)  Step I takes the block residual at Z_t, the point the
      update of Alg. 6 steps from (standard accelerated sketch-and-project);
      point='w' takes it at W_t as Alg. 2 prints.  nesterov='standard'
      (default) forms Z_{t+1} from V_{t+1}; nesterov='literal' uses V_t as
      Alg. 6 prints.  With mu = nu = 1 the standard pair reduces exactly to
      plain SAP with stepsize eta (W = V = Z every step).
  Omega                Gaussian test matrix, orthonormalised by a thin QR
      (Q with a positive-diagonal R), as the commented-out first lines of
      Alg. 4 do.  The Nystrom approximation itself is invariant under
      Omega -> Omega R, but the shift Delta * Omega^T Omega only dominates the
      rounding of a single-precision sketch in every direction when Omega has
      orthonormal columns.
  Alg. 4, line "B <- Y C^{-1}"   Y is the shifted sketch Y_nu = M Omega + Delta Omega.
      "S <- max{0, diag(S^2 - Delta I)}" reads S = max(0, Sigma^2 - Delta).
  eps                  eps of the precision the sketch M Omega is computed in
      (FP32 on the GPU path, as in the paper's single-precision runs):
      2^-23.  Configurable.
  Cholesky failure     (not in the paper) retry with Delta * 10, at most 3 times.
  rho = S_rr + lambda  S_rr is the smallest entry of S (after the clip at 0).
  Alg. 5 final line    lambda <- v_{N-1}^T v_N is read as the Rayleigh quotient
      v_{N-1}^T A v_{N-1} (the unnormalised last product), since the product of
      two normalised vectors is a cosine, not an eigenvalue.
  Stabilised Woodbury with S_i = 0   eigenpairs with S_i = 0 are dropped (the
      limit rho / S_i -> infinity).
  Tail average         W_bar_T = mean(W_j, j = ceil(T/2) .. T).

perturb (tests only; default None, which leaves the arithmetic above exactly as
written): a callback perturb(tag, array) -> array applied to the kernel block
K_BB where a single-precision implementation forms it more than once -- once
for the sketch K_BB Omega (tag "K_BB sketch") and once in the products of the
power iteration (tag "K_BB powering"; for SAP "K_BB solve") -- so that a test
can measure how far rounding of those copies at the FP32 level (Sec. 5 runs in
single precision) moves eta, rho and W.
"""

import numpy as np
import scipy.linalg as sla

from . import kernels as K

EPS_FP32 = 2.0 ** -23


def accel_params(mu, nu):
    """beta, gamma, alpha of Alg. 2 (acceleration parameters)."""
    beta = 1.0 - np.sqrt(mu / nu)
    gamma = 1.0 / np.sqrt(mu * nu)
    alpha = 1.0 / (1.0 + gamma * nu)
    return beta, gamma, alpha


class NystromFailure(RuntimeError):
    pass


def nystrom(Y, Omega, eps=EPS_FP32, retries=3):
    """Alg. 4 (RandNysAppx): from the sketch Y = M Omega and Omega, return (U, S, Delta).

    U (p x r) has orthonormal columns, S (r,) descending, and U diag(S) U^T is
    the rank-r Nystrom approximation of M with the stabilising shift removed.
    """
    Y = np.asarray(Y, dtype=np.float64)
    Omega = np.asarray(Omega, dtype=np.float64)
    OtY = Omega.T @ Y                          # Omega^T M Omega
    OtY = 0.5 * (OtY + OtY.T)                  # symmetric in exact arithmetic
    OtO = Omega.T @ Omega
    Delta = eps * np.trace(OtY)                # shift for stability
    for _ in range(retries + 1):
        H = OtY + Delta * OtO                  # Omega^T M Omega + Delta Omega^T Omega
        try:
            C = np.linalg.cholesky(H).T        # upper: C^T C = H
            break
        except np.linalg.LinAlgError:
            Delta *= 10.0
    else:
        raise NystromFailure("Cholesky of the Nystrom core failed")
    Ynu = Y + Delta * Omega                    # shifted sketch
    # B = Ynu C^{-1}  <=>  C^T B^T = Ynu^T
    B = sla.solve_triangular(C, Ynu.T, trans="T", lower=False).T
    U, Sigma, _ = np.linalg.svd(B, full_matrices=False)   # thin SVD
    S = np.maximum(0.0, Sigma ** 2 - Delta)    # remove the shift
    return U, S, Delta


def orthonormalize(Omega):
    """Thin QR of the test matrix: Q with orthonormal columns, R with positive diagonal."""
    Q, R = np.linalg.qr(np.asarray(Omega, dtype=np.float64))
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    return Q * sgn


def damping(S, lam):
    """rho = S_rr + lambda (Alg. 2, Step III)."""
    return float(np.min(S)) + lam


def woodbury_inv_plain(U, S, rho, g):
    """(U S U^T + rho I)^{-1} g by eq. inv_nys_woodbury (App. C.2)."""
    Utg = U.T @ g
    scale = 1.0 / (S + rho)
    Utg_s = Utg * (scale[:, None] if Utg.ndim == 2 else scale)
    return U @ Utg_s + (g - U @ Utg) / rho


def woodbury_inv_stable(U, S, rho, g):
    """(U S U^T + rho I)^{-1} g via the Cholesky factor L L^T = rho S^{-1} + U^T U (App. C.2)."""
    keep = S > 0
    Uk = U[:, keep]
    Sk = S[keep]
    if Uk.shape[1] == 0:
        return g / rho
    Mcore = np.diag(rho / Sk) + Uk.T @ Uk
    L = np.linalg.cholesky(Mcore)
    y = sla.solve_triangular(L, Uk.T @ g, lower=True)
    y = sla.solve_triangular(L.T, y, lower=False)
    return g / rho - (Uk @ y) / rho


def woodbury_inv_sqrt(U, S, rho, v):
    """(U S U^T + rho I)^{-1/2} v by eq. inv_sqrt_nys_woodbury (App. C.2)."""
    Utv = U.T @ v
    scale = 1.0 / np.sqrt(S + rho)
    Utv_s = Utv * (scale[:, None] if Utv.ndim == 2 else scale)
    return U @ Utv_s + (v - U @ Utv) / np.sqrt(rho)


def get_stepsize(H_mv, Pinvsqrt_mv, v0, N=10):
    """Alg. 5 (GetStepsize): 1 / lambda_1(P^{-1/2} H P^{-1/2}) by randomized powering.

    Returns (eta, lam_hat).
    """
    v = np.asarray(v0, dtype=np.float64)
    v = v / np.linalg.norm(v)
    lam_hat = None
    for i in range(N):
        w = Pinvsqrt_mv(v)
        w = H_mv(w)
        w = Pinvsqrt_mv(w)
        if i == N - 1:
            lam_hat = float(v @ w)             # Rayleigh quotient v_{N-1}^T A v_{N-1}
        v = w / np.linalg.norm(w)
    return 1.0 / lam_hat, lam_hat


def nesterov_acc(W, V, Z, D, eta, beta, gamma, alpha, variant="standard"):
    """Alg. 6 (NesterovAcc); D is the full n x s direction I_B^T D_B."""
    W1 = Z - eta * D
    V1 = beta * V + (1.0 - beta) * Z - gamma * eta * D
    Vz = V if variant == "literal" else V1
    Z1 = alpha * Vz + (1.0 - alpha) * W1
    return W1, V1, Z1


def block_residual(X, Y, P, rows, kernel, ell, sigma2, lam):
    """K_Bn P + lambda I_B P - Y_B (Step I; P is the point the residual is taken at)."""
    return (K.kernel_rows(X, rows, P, kernel, ell, sigma2)
            + lam * P[rows] - Y[rows])


def adasap(X, Y, kernel, ell, sigma2, lam, b, r, T, schedule, W0=None,
           mu=None, nu=None, precond="nystrom", point="z", nesterov="standard",
           eps=EPS_FP32, power_iters=10, tail_average=False, record=None, perturb=None):
    """Alg. 2 (ADASAP) for (K + lambda I) W = Y.

    schedule(t) -> (B_t, Omega_t, v0_t) supplies the iteration's randomness.
    precond: 'nystrom' (ADASAP) or 'identity' (ADASAP-I, P_B = I).
    record: optional list; per iteration a dict of the intermediate results
    (B, R, eta, rho, D_B, ...) is appended.
    Returns W_T (or the tail average).
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    vec = Y.ndim == 1
    Y2 = Y[:, None] if vec else Y
    n = X.shape[0]
    mu = lam if mu is None else mu
    nu = n / b if nu is None else nu
    beta, gamma, alpha = accel_params(mu, nu)
    W = np.zeros_like(Y2) if W0 is None else np.array(W0, dtype=np.float64).reshape(Y2.shape)
    V = W.copy()
    Z = W.copy()
    hist = [W.copy()] if tail_average else None
    for t in range(T):
        Bt, Omega, v0 = schedule(t)
        Bt = np.asarray(Bt)
        # Step I: K_Bn W_t  (at the point chosen by the reading)
        Pt = Z if point == "z" else W
        R = block_residual(X, Y2, Pt, Bt, kernel, ell, sigma2, lam)
        XB = X[Bt]
        KBB = K.kernel_matrix(XB, XB, kernel, ell, sigma2)
        KBB_pow = KBB if perturb is None else perturb("K_BB powering", KBB)
        H_mv = lambda v: KBB_pow @ v + lam * v
        if precond == "nystrom":
            # Step II: Nystrom sketch K_BB Omega (Omega orthonormalised)
            Omega = orthonormalize(Omega)
            MOmega = (KBB if perturb is None else perturb("K_BB sketch", KBB)) @ Omega
            # Step III: Nystrom approximation, preconditioner, stepsize
            U, S, Delta = nystrom(MOmega, Omega, eps=eps)
            rho = damping(S, lam)
            eta, lam_hat = get_stepsize(H_mv, lambda v: woodbury_inv_sqrt(U, S, rho, v),
                                        v0, N=power_iters)
            # Step IV: search direction P_B^{-1} R
            DB = woodbury_inv_stable(U, S, rho, R)
        elif precond == "identity":
            U = S = Delta = rho = None
            eta, lam_hat = get_stepsize(H_mv, lambda v: v, v0, N=power_iters)
            DB = R.copy()
        else:
            raise ValueError(precond)
        D = np.zeros_like(W)
        D[Bt] = DB
        W, V, Z = nesterov_acc(W, V, Z, D, eta, beta, gamma, alpha, variant=nesterov)
        if tail_average:
            hist.append(W.copy())
        if record is not None:
            record.append(dict(B=Bt, R=R, eta=eta, lam_hat=lam_hat, rho=rho,
                               Delta=Delta, S=S, U=U, D_B=DB, W=W.copy(), Z=Z.copy()))
    if tail_average:
        Tn = len(hist) - 1
        out = np.mean(hist[(Tn + 1) // 2:], axis=0)
    else:
        out = W
    return out[:, 0] if vec else out


def sap(X, Y, kernel, ell, sigma2, lam, b, T, blocks, W0=None, tail_average=False, perturb=None):
    """Alg. 1 (SAP) with the exact block solve (K_BB + lambda I)^{-1}.

    blocks(t) -> B_t.  Returns W_T (or the tail average).
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    vec = Y.ndim == 1
    Y2 = Y[:, None] if vec else Y
    W = np.zeros_like(Y2) if W0 is None else np.array(W0, dtype=np.float64).reshape(Y2.shape)
    hist = [W.copy()]
    for t in range(T):
        Bt = np.asarray(blocks(t))
        R = block_residual(X, Y2, W, Bt, kernel, ell, sigma2, lam)
        XB = X[Bt]
        KBB = K.kernel_matrix(XB, XB, kernel, ell, sigma2)
        Hb = (KBB if perturb is None else perturb("K_BB solve", KBB)) + lam * np.eye(len(Bt))
        DB = sla.cho_solve(sla.cho_factor(Hb), R)
        W = W.copy()
        W[Bt] -= DB
        hist.append(W.copy())
    if tail_average:
        Tn = len(hist) - 1
        out = np.mean(hist[(Tn + 1) // 2:], axis=0)
    else:
        out = W
    return out[:, 0] if vec else out
