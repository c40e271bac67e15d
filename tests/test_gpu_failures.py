"""Failure detection on the GPU without a fault: a bounded wait that runs out,
and a diverging solve, are reported as statuses, and the context stays usable."""

import numpy as np
import pytest
import torch

from oracle import kernels as OK
from paper_2505_13723_b300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_is_reported(lib):
    """A wait that nothing completes gives up after its limit (1 ms here), records its
    code, and the next kernels of the same context run normally."""
    P = synth.small(n=800)
    ctx = lib.Context(P.X, P.kernel, P.ell, P.sigma2, P.lam)
    assert ctx.check_device() == (0, 0)
    ctx.wait_selftest(1_000_000)
    assert ctx.check_device() == (6, 99)          # ADASAP_ETIMEOUT, the self-test's code
    assert ctx.check_device() == (0, 0)           # the record is cleared by the check
    rows = np.arange(0, 800, 5)
    W = np.random.default_rng(1).standard_normal((800, 1)).astype(np.float32)
    out = ctx.kernel_rows(torch.from_numpy(rows).cuda(), torch.from_numpy(W).cuda()).cpu().numpy()
    Xd = P.X.astype(np.float64)
    ref = OK.kernel_apply(Xd[rows], Xd, W.astype(np.float64), P.kernel, P.ell, P.sigma2)
    scale = OK.kernel_apply(Xd[rows], Xd, np.abs(W.astype(np.float64)), P.kernel, P.ell, P.sigma2)
    assert (np.abs(out - ref) <= 1e-5 * scale).all()
    assert ctx.check_device() == (0, 0)


def test_nan_in_y_is_reported_as_divergence(lib):
    """A NaN in the right-hand side makes the iterate non-finite: the residual check
    returns a failure status (EDIVERGED, or ENUMERIC if a factorisation saw it first)
    instead of a result, and a clean solve on the same context then succeeds."""
    P = synth.small(n=1000)
    n = P.X.shape[0]
    ctx = lib.Context(P.X, P.kernel, P.ell, P.sigma2, P.lam)
    Y = P.Y.copy()
    Y[17, 0] = np.nan
    opts = lib.default_opts(n, b=100, r=20, max_iters=6, check_every=2, seed=3)
    with pytest.raises(lib.AdasapError) as err:
        ctx.solve(torch.from_numpy(Y).cuda(), opts=opts)
    assert err.value.status in (4, 5)
    W, st, status = ctx.solve(torch.from_numpy(P.Y).cuda(), opts=opts)
    assert status == 0 and np.isfinite(W.cpu().numpy()).all() and st["rel_resid"] < 1.0
