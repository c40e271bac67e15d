"""GPU parity of adasap_solve_batched (many independent systems of uneven n in
one graph, grouped tensor-core launches) against the FP64 oracle.

Each system runs Alg. 2 with its own device randomness (Philox keyed by its
seed); the oracle replays the same counter-based draws.  The grouped launch
changes only the column split of the Step I and K_BB a sums (rounding order),
so the per-system tolerance is the one of the single-system parity tests
(tests/_parity.py): 10x the oracle's own sensitivity to FP32-level rounding of
X and Omega, capped by max(1e-4, (2N + 1) * 4 * 2^-23 * b * sigma2 / min_t rho_t).
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


def _systems(count, nmin, nmax, seed, lam=1e-2):
    out = []
    for P in synth.bo_systems(count=count, nmin=nmin, nmax=nmax, seed=seed):
        n = P.X.shape[0]
        P["b"] = max(n // 10, 40)
        P["r"] = 20
        P["lam"] = lam
        out.append(P)
    return out


def _oracle(P, T, seed, precond="nystrom", Y=None):
    """The oracle's W_T and its sensitivity (tests/_parity.py) for one system."""
    n = P.X.shape[0]
    Yd = (P.Y if Y is None else Y).astype(np.float64)

    def run(Xp, sched, hook):
        rec = []
        W = OA.adasap(Xp, Yd, P.kernel, P.ell, P.sigma2, P.lam, P.b, P.r, T, sched, precond=precond, record=rec,
                      perturb=hook)
        return W, rec

    return PT.sensitivity(run, P.X, OR.philox_schedule(n, P.b, P.r, seed=seed), seed=seed)


def _check_w(name, W, Wref, rec, sens, P):
    PT.check(name, [("W", _rel(W, Wref), sens["W"], PT.a_priori_cap(rec, P.b, P.sigma2))])


def test_batched_uneven_systems_match_oracle(lib):
    """Five Matern-5/2 systems, n from ~400 to ~3000, d in {4, 8, 12}: every system's
    W_T after 5 iterations against the oracle, and against its own single-system solve."""
    Ps = _systems(5, 400, 3000, seed=11)
    T = 5
    ctxs = [lib.Context(P.X, P.kernel, P.ell, P.sigma2, P.lam) for P in Ps]
    opts = [lib.default_opts(P.X.shape[0], b=P.b, r=P.r, max_iters=T, check_every=0, seed=100 + k)
            for k, P in enumerate(Ps)]
    Ws, stats, status = lib.solve_batched(ctxs, [torch.from_numpy(P.Y).cuda() for P in Ps], opts=opts)
    assert status == 0
    for k, (P, ctx, W, st) in enumerate(zip(Ps, ctxs, Ws, stats)):
        assert st["iters"] == T and st["resid_exact"] == 1
        Wref, rec, sens = _oracle(P, T, 100 + k)
        _check_w("batched uneven k=%d" % k, W.cpu().numpy(), Wref, rec, sens, P)
        # same system alone (same seed): equal up to the rounding order of the split sums
        Wone, _, _ = ctx.solve(torch.from_numpy(P.Y).cuda(), opts=opts[k])
        PT.check("batched vs alone k=%d" % k, [("W", _rel(W.cpu().numpy(), Wone.cpu().numpy()), sens["W"],
                                                PT.a_priori_cap(rec, P.b, P.sigma2))])
        # the reported residual is the exact one of the returned W
        ref = gp.rel_residual(P.X.astype(np.float64), W.cpu().numpy(), P.Y, P.kernel, P.ell, P.sigma2, P.lam)
        assert abs(st["rel_resid"] - ref) <= 1e-3 * ref


def test_batched_mixed_members(lib):
    """Systems that cannot join the grouped launches (identity preconditioner, FP32
    CUDA-core precision) iterate in the same graph as grouped ones, and the grouped ones
    form several classes (an RBF kernel; d = 20, whose operands are 32 wide)."""
    Ps = _systems(5, 500, 2000, seed=12)
    Ps[2]["kernel"] = synth.RBF
    rng = np.random.default_rng(12)
    Ps[4]["X"] = rng.uniform(-1.0, 1.0, (Ps[4].X.shape[0], 20)).astype(np.float32)
    T = 4
    ctxs = [lib.Context(P.X, P.kernel, P.ell, P.sigma2, P.lam) for P in Ps]
    ctxs[1].set_precision(lib.PREC_FP32)
    opts = [lib.default_opts(P.X.shape[0], b=P.b, r=P.r, max_iters=T, check_every=0, seed=200 + k)
            for k, P in enumerate(Ps)]
    opts[3].precond = 1
    Ws, stats, status = lib.solve_batched(ctxs, [P.Y for P in Ps], opts=opts)
    assert status == 0 and all(isinstance(W, np.ndarray) for W in Ws)
    for k, (P, W) in enumerate(zip(Ps, Ws)):
        Wref, rec, sens = _oracle(P, T, 200 + k, precond="identity" if k == 3 else "nystrom")
        _check_w("batched mixed k=%d" % k, W, Wref, rec, sens, P)


def test_batched_systems_leave_at_their_tolerance(lib):
    """Well-conditioned systems converge after different iteration counts; each leaves
    the batch at its first check below tol (the graph is re-captured without it)."""
    Ps = _systems(4, 300, 1500, seed=13, lam=0.3)
    ctxs = [lib.Context(P.X, P.kernel, P.ell, P.sigma2, P.lam) for P in Ps]
    opts = [lib.default_opts(P.X.shape[0], b=P.b, r=P.r, max_iters=1000, tol=1e-5, check_every=5,
                             seed=300 + k) for k, P in enumerate(Ps)]
    Ws, stats, status = lib.solve_batched(ctxs, [torch.from_numpy(P.Y).cuda() for P in Ps], opts=opts)
    assert status == 0, stats
    iters = [st["iters"] for st in stats]
    for P, W, st in zip(Ps, Ws, stats):
        assert st["rel_resid"] <= 1e-5 and st["iters"] % 5 == 0 and st["iters"] < 1000
        Wstar = gp.solve_dense(P.X.astype(np.float64), P.Y.astype(np.float64), P.kernel, P.ell, P.sigma2, P.lam)
        assert _rel(W.cpu().numpy(), Wstar) < 1e-3
    assert len(set(iters)) > 1, iters


def test_batched_invalid_arguments(lib):
    Ps = _systems(2, 300, 400, seed=14)
    ctx = lib.Context(Ps[0].X, Ps[0].kernel, Ps[0].ell, Ps[0].sigma2, Ps[0].lam)
    o = lib.default_opts(Ps[0].X.shape[0], b=Ps[0].b, r=Ps[0].r, max_iters=2)
    with pytest.raises(lib.AdasapError):
        lib.solve_batched([ctx, ctx], [Ps[0].Y, Ps[0].Y], opts=[o, o])
    o2 = lib.default_opts(Ps[0].X.shape[0], b=Ps[0].b, r=Ps[0].r, max_iters=2, tail_average=1)
    with pytest.raises(lib.AdasapError):
        lib.solve_batched([ctx], [Ps[0].Y], opts=[o2])


def test_batched_requires_one_powering_length(lib):
    Ps = _systems(2, 300, 400, seed=15)
    ctxs = [lib.Context(P.X, P.kernel, P.ell, P.sigma2, P.lam) for P in Ps]
    opts = [lib.default_opts(P.X.shape[0], b=P.b, r=P.r, max_iters=2, power_iters=10 + k) for k, P in enumerate(Ps)]
    with pytest.raises(lib.AdasapError):
        lib.solve_batched(ctxs, [P.Y for P in Ps], opts=opts)


def test_batched_multi_rhs_members(lib):
    """s = 2: no member joins the grouped single-RHS launches; every system's own
    multi-RHS path runs inside the batch graph."""
    Ps = _systems(3, 400, 1500, seed=16)
    T = 3
    rng = np.random.default_rng(16)
    Ys = [np.concatenate([P.Y, rng.standard_normal((P.X.shape[0], 1)).astype(np.float32)], axis=1) for P in Ps]
    ctxs = [lib.Context(P.X, P.kernel, P.ell, P.sigma2, P.lam) for P in Ps]
    opts = [lib.default_opts(P.X.shape[0], b=P.b, r=P.r, max_iters=T, check_every=0, seed=500 + k)
            for k, P in enumerate(Ps)]
    Ws, stats, status = lib.solve_batched(ctxs, [torch.from_numpy(Y).cuda() for Y in Ys], opts=opts)
    assert status == 0
    for k, (P, Y, W) in enumerate(zip(Ps, Ys, Ws)):
        Wref, rec, sens = _oracle(P, T, 500 + k, Y=Y)
        _check_w("batched s=2 k=%d" % k, W.cpu().numpy(), Wref, rec, sens, P)


def test_batched_bo_workload_full_size(lib):
    """The 48-system bo workload as benchmarked (n log-uniform in [4096, 65536], b = n/50,
    r = 50), two iterations: every system finishes with status 0 and a finite residual, and
    the two smallest systems match the oracle's replay of their device randomness."""
    Ps = synth.bo_systems()
    T = 2
    ctxs = [lib.Context(torch.from_numpy(P.X).cuda(), P.kernel, P.ell, P.sigma2, P.lam) for P in Ps]
    opts = [lib.default_opts(P.X.shape[0], b=P.b, r=P.r, max_iters=T, check_every=0, check_rows=4096,
                             seed=40 + k) for k, P in enumerate(Ps)]
    Ws, stats, status = lib.solve_batched(ctxs, [torch.from_numpy(P.Y).cuda() for P in Ps], opts=opts)
    assert status == 0
    assert all(st["iters"] == T and np.isfinite(st["rel_resid"]) for st in stats)
    for k in np.argsort([P.X.shape[0] for P in Ps])[:2]:
        P = Ps[k]
        Wref, rec, sens = _oracle(P, T, 40 + int(k))
        _check_w("bo full-size k=%d n=%d" % (k, P.X.shape[0]), Ws[k].cpu().numpy(), Wref, rec, sens, P)


def test_batched_bo_workload_repeats_bit_for_bit(lib):
    """The grouped tensor-core launches let each CTA take its next item from a shared
    counter, so which CTA computes an item depends on timing; an item's result must
    not (its partial sums are combined in a fixed order).  Two solves of the 48-system
    bo workload with the same inputs and seeds give the same W, bit for bit."""
    Ps = synth.bo_systems()
    ctxs = [lib.Context(torch.from_numpy(P.X).cuda(), P.kernel, P.ell, P.sigma2, P.lam) for P in Ps]
    Ys = [torch.from_numpy(P.Y).cuda() for P in Ps]
    out = []
    for _ in range(2):
        opts = [lib.default_opts(P.X.shape[0], b=P.b, r=P.r, max_iters=3, check_every=0, check_rows=4096,
                                 seed=40 + k) for k, P in enumerate(Ps)]
        Ws, stats, status = lib.solve_batched(ctxs, Ys, opts=opts)
        assert status == 0
        out.append([W.cpu().numpy() for W in Ws])
    for k, (a, b) in enumerate(zip(*out)):
        assert np.array_equal(a, b), "system %d differs between two identical solves" % k
