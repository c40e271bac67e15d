"""GPU parity of SAP with the exact block solve (Alg. 1; opts.precond = 2) against
the FP64 oracle.

The GPU forms H = K_BB + lambda I from the FP32 centred, scaled points, so its
entries differ from the oracle's by ~2^-23 relative; the direction H^{-1} R then
moves by up to cond(H) times that.  cond(H) <= (b sigma2 + lambda) / lambda, so the
a-priori bound is  max(1e-4, 10 * 2^-23 * (b sigma2 + lambda) / lambda).  The
blocked FP32 Cholesky's own rounding is removed by two refinement steps (residual
R - H D in FP64), which the one-block test checks against the GPU's own residual.
The W_T checks against the oracle's Alg. 1 use 10x the oracle's own sensitivity
to FP32-level rounding of the points X (tests/_parity.py), with that bound as the
cap.
"""

import numpy as np
import pytest
import torch

from oracle import adasap as OA
from oracle import gp
from oracle import rng as OR
from paper_2505_13723_b300 import synth

import _parity as PT

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _tol(b, sigma2, lam):
    return max(1e-4, 10 * 2.0 ** -23 * (b * sigma2 + lam) / lam)


@pytest.mark.parametrize("kern,b,T,tail", [(0, 150, 5, False), (1, 333, 4, False), (2, 64, 6, True),
                                           (0, 1000, 2, False)])
def test_sap_exact_matches_oracle(lib, kern, b, T, tail):
    P = synth.small(n=1500)
    n = P.X.shape[0]
    lam = 0.1
    ctx = lib.Context(P.X, kern, P.ell, P.sigma2, lam)
    opts = lib.default_opts(n, b=b, precond=2, max_iters=T, check_every=0, seed=5 + b, tail_average=int(tail))
    W, st, status = ctx.solve(torch.from_numpy(P.Y).cuda(), opts=opts)
    assert status == 0 and st["iters"] == T
    Yd = P.Y.astype(np.float64)

    def run(Xp, _, hook):
        return OA.sap(Xp, Yd, kern, P.ell, P.sigma2, lam, b, T, lambda t: OR.sample_block(n, b, 5 + b, t),
                      tail_average=tail, perturb=hook), []

    Wref, _, sens = PT.sensitivity(run, P.X, None, seed=b)
    PT.check("sap kern=%d b=%d T=%d" % (kern, b, T), [("W", _rel(W.cpu().numpy(), Wref), sens["W"],
                                                        _tol(b, P.sigma2, lam))])


def test_sap_exact_one_block_is_the_solution(lib):
    """b = n (ragged against the 64-row tiles): one step from W_0 = 0 solves the system
    (the oracle's Cholesky solution, and the GPU's own exact residual)."""
    P = synth.small(n=700, d=5)
    n = P.X.shape[0]
    lam = 0.3
    ctx = lib.Context(P.X, 2, P.ell, P.sigma2, lam)
    opts = lib.default_opts(n, b=n, precond=2, max_iters=1, check_every=0, seed=1)
    W, st, status = ctx.solve(torch.from_numpy(P.Y).cuda(), opts=opts)
    assert status == 0
    Wstar = gp.solve_dense(P.X.astype(np.float64), P.Y.astype(np.float64), 2, P.ell, P.sigma2, lam)
    assert _rel(W.cpu().numpy(), Wstar) < _tol(n, P.sigma2, lam)
    # against the GPU's own operator the refined solve is at the FP32 rounding level
    assert st["rel_resid"] < 1e-5 and ctx.residual(torch.from_numpy(P.Y).cuda(), W) < 1e-5


def test_sap_exact_multi_rhs_large_block(lib):
    """b = 2048 (32 tiles, 32 panels of the blocked Cholesky), s = 3, two iterations."""
    P = synth.multirhs(n=4096, s=3, b=2048)
    n = P.X.shape[0]
    lam = 0.5
    ctx = lib.Context(P.X, P.kernel, P.ell, P.sigma2, lam)
    opts = lib.default_opts(n, b=2048, precond=2, max_iters=2, check_every=0, seed=8)
    W, st, status = ctx.solve(torch.from_numpy(P.Y).cuda(), opts=opts)
    assert status == 0
    Yd = P.Y.astype(np.float64)

    def run(Xp, _, hook):
        return OA.sap(Xp, Yd, P.kernel, P.ell, P.sigma2, lam, 2048, 2, lambda t: OR.sample_block(n, 2048, 8, t),
                      perturb=hook), []

    Wref, _, sens = PT.sensitivity(run, P.X, None, seed=8)
    PT.check("sap b=2048 s=3", [("W", _rel(W.cpu().numpy(), Wref), sens["W"], _tol(2048, P.sigma2, lam))])


def test_sap_exact_converges_and_batch_refuses_it(lib):
    P = synth.small(n=1000, d=3)
    n = P.X.shape[0]
    ctx = lib.Context(P.X, 0, P.ell, P.sigma2, 0.3)
    opts = lib.default_opts(n, b=250, precond=2, max_iters=600, tol=1e-5, check_every=5, seed=2)
    W, st, status = ctx.solve(torch.from_numpy(P.Y).cuda(), opts=opts)
    assert status == 0 and st["rel_resid"] <= 1e-5
    Wstar = gp.solve_dense(P.X.astype(np.float64), P.Y.astype(np.float64), 0, P.ell, P.sigma2, 0.3)
    assert _rel(W.cpu().numpy(), Wstar) < 1e-3
    with pytest.raises(lib.AdasapError):
        lib.solve_batched([ctx], [P.Y], opts=[opts])
