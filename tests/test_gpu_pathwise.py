"""GPU parity of the pathwise-conditioning path (Sec. 2.1): random-feature prior
draws, posterior samples through the s-column ADASAP solve, test RMSE / NLL.

Tolerance of the prior draws.  Each feature term is theta * cos(arg) with
|arg| <= A; the FP32 argument carries a rounding error of a few ulps of A, the
cosine one ulp, and the q-term FP32 sum a relative error of at most about
q * 2^-24 of the sum of absolute terms (recursive summation).  So each entry is
held to  (q * 2^-24 + 4e-7 * (1 + A)) * sqrt(2 sigma2 / q) * sum_l |theta_l|.

The posterior samples after a few ADASAP iterations are held to 10x the
oracle's own sensitivity to FP32-level rounding of X and Omega
(tests/_parity.py), capped by the solver tests' a-priori bound.
"""

import numpy as np
import pytest
import torch

from oracle import adasap as OA
from oracle import gp
from oracle import kernels as OK
from oracle import pathwise as PW
from oracle import rng as OR
from paper_2505_13723_b300 import synth

import _parity as PT

pytestmark = pytest.mark.gpu

DOF = {0: None, 1: 3, 2: 5}   # chi^2 degrees of freedom 2 nu of the Matern spectral draws


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _cuda(*arrs):
    return [torch.from_numpy(a).cuda() if a is not None else None for a in arrs]


@pytest.mark.parametrize("kern,d,m,q,s", [(0, 3, 1000, 2048, 1), (1, 11, 777, 1000, 4), (2, 8, 1531, 2048, 64),
                                          (0, 16, 300, 333, 100), (1, 40, 200, 128, 9), (2, 1, 65, 64, 17)])
def test_rf_prior_matches_oracle(lib, kern, d, m, q, s):
    rng = np.random.default_rng(kern * 100 + d)
    # the context's points have a mean far from 0: the centring is undone in the phase
    X = (rng.random((500, d)) + 3.0).astype(np.float32)
    Xq = (rng.random((m, d)) * 2.0 + 2.0).astype(np.float32)
    ell, sigma2 = 0.7, 1.7
    z, u, phase, theta, _ = synth.rf_draws(q, d, DOF[kern], s, 1, 1.0, seed=d + s)
    ctx = lib.Context(X, kern, ell, sigma2, 1e-2)
    F = ctx.rf_prior(*_cuda(Xq, z, u, phase, theta)).cpu().numpy()
    ref = PW.rf_prior(Xq, z, u, phase, theta, kern, ell, sigma2)
    omega = PW.rf_frequencies(z, u, kern, ell)
    A = np.abs(Xq.astype(np.float64) @ omega.T + phase.astype(np.float64)).max()
    bound = (q * 2.0 ** -24 + 4e-7 * (1.0 + A)) * np.sqrt(2 * sigma2 / q) * np.abs(theta).astype(np.float64).sum(0)
    assert np.isfinite(F).all()
    assert (np.abs(F - ref) <= bound[None, :]).all(), np.abs(F - ref).max()


def _pathwise_case(lib, P, ns, T, seed, kern=None, prec=None):
    kern = P.kernel if kern is None else kern
    n, d = P.X.shape
    q = 512
    z, u, phase, theta, zeta = synth.rf_draws(q, d, DOF[kern], ns, n, P.lam, seed=seed)
    ctx = lib.Context(P.X, kern, P.ell, P.sigma2, P.lam, precision=prec)
    y = P.Y[:, 0].copy()
    opts = lib.default_opts(n, b=P.b, r=P.r, max_iters=T, check_every=0, seed=seed)
    out, W, st, status = ctx.pathwise(*_cuda(y, P.Xtest, z, u, phase, theta, zeta), opts=opts)
    Xt = P.Xtest.astype(np.float64)

    def run(Xd, sched, hook):
        FX = PW.rf_prior(Xd, z, u, phase, theta, kern, P.ell, P.sigma2)
        Fs = PW.rf_prior(Xt, z, u, phase, theta, kern, P.ell, P.sigma2)
        R = np.concatenate([y.astype(np.float64)[:, None], PW.pathwise_rhs(y, FX, zeta)], axis=1)
        rec = []
        Wref = OA.adasap(Xd, R, kern, P.ell, P.sigma2, P.lam, P.b, P.r, T, sched, record=rec, perturb=hook)
        out_ref = np.concatenate([gp.posterior_mean(Xt, Xd, Wref[:, :1], kern, P.ell, P.sigma2),
                                  PW.pathwise_samples(Xt, Xd, Wref[:, 1:], Fs, kern, P.ell, P.sigma2)], axis=1)
        # W and the samples together, so that the sensitivity covers both
        return (Wref, out_ref), rec

    sens_all = {}

    def run_flat(Xd, sched, hook):
        (Wr, outr), rec = run(Xd, sched, hook)
        sens_all.setdefault("runs", []).append((Wr, outr))
        return np.concatenate([Wr.ravel(), outr.ravel()]), rec

    _, rec, _ = PT.sensitivity(run_flat, P.X, OR.philox_schedule(n, P.b, P.r, seed=seed), seed=seed)
    (Wref, out_ref), pert = sens_all["runs"][0], sens_all["runs"][1:]
    sens = {"W": max(PT.rel(a, Wref) for a, _ in pert), "out": max(PT.rel(b, out_ref) for _, b in pert)}
    return out.cpu().numpy(), W.cpu().numpy(), out_ref, Wref, rec, sens, status


@pytest.mark.parametrize("kern,prec", [(0, None), (1, None), (2, 0)])
def test_pathwise_samples_match_oracle(lib, kern, prec):
    """Seven samples plus the mean through 6 ADASAP iterations (device randomness, replayed
    by the oracle): W and the samples at 500 test points; the last case on the FP32
    CUDA-core path."""
    P = synth.small(n=1500)
    out, W, out_ref, Wref, rec, sens, status = _pathwise_case(lib, P, ns=7, T=6, seed=17 + kern, kern=kern,
                                                              prec=prec)
    assert status == 0
    cap = PT.a_priori_cap(rec, P.b, P.sigma2)
    PT.check("pathwise kern=%d prec=%s" % (kern, prec), [("W", _rel(W, Wref), sens["W"], cap),
                                                         ("samples", _rel(out, out_ref), sens["out"], cap)])


def test_pathwise_converged_matches_cholesky(lib):
    """A converged solve gives the samples of eq. pathwise_conditoning with a Cholesky solve."""
    P = synth.small(n=1200, d=3)
    P["lam"] = 0.3
    n, d = P.X.shape
    ns, q = 5, 256
    z, u, phase, theta, zeta = synth.rf_draws(q, d, None, ns, n, P.lam, seed=3)
    ctx = lib.Context(P.X, 0, P.ell, P.sigma2, P.lam)
    y = P.Y[:, 0].copy()
    opts = lib.default_opts(n, b=300, r=64, max_iters=2000, tol=1e-5, check_every=10, seed=4)
    out, W, st, status = ctx.pathwise(*_cuda(y, P.Xtest, z, u, phase, theta, zeta), opts=opts)
    assert status == 0 and st["rel_resid"] <= 1e-5, st
    Xd, Xt = P.X.astype(np.float64), P.Xtest.astype(np.float64)
    FX = PW.rf_prior(Xd, z, u, phase, theta, 0, P.ell, P.sigma2)
    Fs = PW.rf_prior(Xt, z, u, phase, theta, 0, P.ell, P.sigma2)
    ref = PW.pathwise_exact(Xt, Xd, y, FX, Fs, zeta, 0, P.ell, P.sigma2, P.lam)
    mean_ref = gp.posterior_mean(Xt, Xd, gp.solve_dense(Xd, y[:, None], 0, P.ell, P.sigma2, P.lam), 0, P.ell,
                                 P.sigma2)
    out = out.cpu().numpy()
    # rel-resid 1e-5 with lambda = 0.3 moves W by at most ||r|| / lambda: the samples agree to ~1e-4
    assert _rel(out[:, 1:], ref) < 1e-3
    assert _rel(out[:, :1], mean_ref) < 1e-3


def test_pathwise_single_sample_without_mean(lib):
    P = synth.small(n=700, d=4)
    n, d = P.X.shape
    z, u, phase, theta, zeta = synth.rf_draws(128, d, 5, 1, n, P.lam, seed=9)
    ctx = lib.Context(P.X, 2, P.ell, P.sigma2, P.lam)
    y = P.Y[:, 0].copy()
    opts = lib.default_opts(n, b=70, r=20, max_iters=3, check_every=0, seed=9)
    out, W, st, status = ctx.pathwise(*_cuda(y, P.Xtest, z, u, phase, theta, zeta), with_mean=False, opts=opts)
    Xd, Xt = P.X.astype(np.float64), P.Xtest.astype(np.float64)
    FX = PW.rf_prior(Xd, z, u, phase, theta, 2, P.ell, P.sigma2)
    Fs = PW.rf_prior(Xt, z, u, phase, theta, 2, P.ell, P.sigma2)
    rhs = PW.pathwise_rhs(y, FX, zeta)

    def run(Xp, sched, hook):
        rec = []
        Wr = OA.adasap(Xp, rhs, 2, P.ell, P.sigma2, P.lam, 70, 20, 3, sched, record=rec, perturb=hook)
        return PW.pathwise_samples(Xt, Xp, Wr, Fs, 2, P.ell, P.sigma2), rec

    ref, rec, sens = PT.sensitivity(run, Xd, OR.philox_schedule(n, 70, 20, seed=9), seed=9)
    assert out.shape == (P.Xtest.shape[0], 1)
    PT.check("pathwise one sample", [("samples", _rel(out.cpu().numpy(), ref), sens["W"],
                                      PT.a_priori_cap(rec, 70, P.sigma2))])
    # a Matern context without its chi-square draws is refused
    with pytest.raises(lib.AdasapError):
        ctx.rf_prior(*_cuda(P.Xtest, z, None, phase, theta))


def test_rmse_nll_matches_oracle(lib):
    rng = np.random.default_rng(8)
    m, ns = 1003, 16
    out = rng.standard_normal((m, ns + 1)).astype(np.float32)
    yt = (out[:, 0] + 0.3 * rng.standard_normal(m)).astype(np.float32)
    o = torch.from_numpy(out).cuda()
    rm, nl = lib.rmse_nll(o[:, 0], o[:, 1:], torch.from_numpy(yt).cuda(), 0.01)
    rm_ref, nl_ref = PW.rmse_nll(out[:, 0], out[:, 1:], yt, 0.01)
    assert rm == pytest.approx(rm_ref, rel=1e-9) and nl == pytest.approx(nl_ref, rel=1e-9)


def test_rf_prior_multirhs_workload_full_size_sampled(lib):
    """The prior draw the pathwise benchmark times: n = 2^18 training points, q = 2048,
    63 samples; 32 sampled points checked against the oracle."""
    P = synth.multirhs()
    n, d = P.X.shape
    q, ns = 2048, 63
    z, u, phase, theta, _ = synth.rf_draws(q, d, None, ns, 1, P.lam, seed=1)
    ctx = lib.Context(P.X, P.kernel, P.ell, P.sigma2, P.lam)
    F = ctx.rf_prior(*_cuda(P.X, z, u, phase, theta)).cpu().numpy()
    pick = np.random.default_rng(3).choice(n, size=32, replace=False)
    ref = PW.rf_prior(P.X[pick], z, u, phase, theta, P.kernel, P.ell, P.sigma2)
    omega = PW.rf_frequencies(z, u, P.kernel, P.ell)
    A = np.abs(P.X[pick].astype(np.float64) @ omega.T + phase.astype(np.float64)).max()
    bound = (q * 2.0 ** -24 + 4e-7 * (1.0 + A)) * np.sqrt(2 * P.sigma2 / q) * np.abs(theta).astype(np.float64).sum(0)
    assert (np.abs(F[pick] - ref) <= bound[None, :]).all()
