"""Seeded synthetic workloads for the ADASAP hot path.

This module only draws data.  It holds none of the solver's arithmetic, so both
the CUDA path's tests/bench and the FP64 oracle may read it.

The paper's datasets (Table 1, the taxi data of Sec. 5.2, the BO problems of
Sec. 5.3) are not available here; these generators stand in for them with the
same shapes, dimensions, kernels and hyperparameter ranges.  All data are drawn
in float64 with numpy.random.default_rng and cast to float32 (the solver's
storage type); the oracle reads the same float32 values upcast to float64.

Workloads
---------
small    n=2000, d=8, X ~ N(0, I), y = sin(2 X u) + 0.1 eps with u a random unit
         vector, RBF ell=1, sigma2=1, lambda=1e-2, b=200, r=32, 300 iterations,
         500 test points, single right-hand side.  Seed 0.
regress  n=2^20, d=11, X ~ U[0,1]^d, y = sum_k sin(3 x_k) + 0.05 eps,
         Matern-3/2 ell=0.3, lambda=1e-3, b=10000, r=100, single RHS.  Seed 2.
multirhs n=2^18, d=16, X ~ N(0, I), Y = [y, 63 columns of N(0,1)] (s=64),
         y = sin(2 X u) + 0.1 eps, RBF ell=2, lambda=1e-2, b=4096, r=64.  Seed 3.
bo       48 independent systems, n log-uniform in [4096, 65536], d in {4, 8, 12},
         X ~ U[-1,1]^d, y = sum_k sin(3 x_k) + 0.05 eps, Matern-5/2
         ell ~ U[0.2, 1], lambda=1e-3, b=n/50, r=50.  Seed 4.
taxi     n=2^25, d=9, X ~ U[0,1]^9, y = sum_k cos(4 x_k) + 0.1 eps, RBF ell=0.5,
         lambda=1e-2, b=100000, r=100, single RHS.  Seed 5.
Test points (where used) are drawn from the training distribution.  Every
generator takes an optional ``n`` to shrink the problem for tests while keeping
the distribution.
"""

import numpy as np

RBF, MATERN32, MATERN52 = 0, 1, 2


class Problem(dict):
    """A workload: X (n,d) f32, Y (n,s) f32, Xtest (m,d) f32 and its hyperparameters."""
    __getattr__ = dict.__getitem__


def _unit_vector(rng, d):
    u = rng.standard_normal(d)
    return u / np.linalg.norm(u)


def small(n=2000, d=8, m=500, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    u = _unit_vector(rng, d)
    y = np.sin(2.0 * X @ u) + 0.1 * rng.standard_normal(n)
    Xt = rng.standard_normal((m, d))
    return Problem(name="small", X=X.astype(np.float32), Y=y[:, None].astype(np.float32),
                   Xtest=Xt.astype(np.float32), kernel=RBF, ell=1.0, sigma2=1.0,
                   lam=1e-2, b=min(200, n), r=32, iters=300)


def regress(n=1 << 20, d=11, m=10000, seed=2, b=None):
    rng = np.random.default_rng(seed)
    X = rng.random((n, d))
    y = np.sin(3.0 * X).sum(axis=1) + 0.05 * rng.standard_normal(n)
    Xt = rng.random((m, d))
    return Problem(name="regress", X=X.astype(np.float32), Y=y[:, None].astype(np.float32),
                   Xtest=Xt.astype(np.float32), kernel=MATERN32, ell=0.3, sigma2=1.0,
                   lam=1e-3, b=b if b is not None else min(10000, n // 4), r=100, iters=None)


def multirhs(n=1 << 18, d=16, m=10000, s=64, seed=3, b=None):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    u = _unit_vector(rng, d)
    y = np.sin(2.0 * X @ u) + 0.1 * rng.standard_normal(n)
    Y = np.concatenate([y[:, None], rng.standard_normal((n, s - 1))], axis=1)
    Xt = rng.standard_normal((m, d))
    return Problem(name="multirhs", X=X.astype(np.float32), Y=Y.astype(np.float32),
                   Xtest=Xt.astype(np.float32), kernel=RBF, ell=2.0, sigma2=1.0,
                   lam=1e-2, b=b if b is not None else min(4096, n // 4), r=64, iters=None)


def bo_systems(count=48, nmin=4096, nmax=65536, seed=4):
    """The uneven batch: a list of Problems (one per independent GP system)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))
        d = int(rng.choice([4, 8, 12]))
        ell = float(rng.uniform(0.2, 1.0))
        X = rng.uniform(-1.0, 1.0, (n, d))
        y = np.sin(3.0 * X).sum(axis=1) + 0.05 * rng.standard_normal(n)
        out.append(Problem(name="bo%02d" % k, X=X.astype(np.float32),
                           Y=y[:, None].astype(np.float32), Xtest=None,
                           kernel=MATERN52, ell=ell, sigma2=1.0, lam=1e-3,
                           b=max(1, n // 50), r=50, iters=None))
    return out


def taxi(n=1 << 25, d=9, m=10000, seed=5, b=None):
    rng = np.random.default_rng(seed)
    X = np.empty((n, d), dtype=np.float32)
    y = np.empty(n, dtype=np.float32)
    step = 1 << 22
    for i0 in range(0, n, step):
        i1 = min(n, i0 + step)
        Xc = rng.random((i1 - i0, d))
        X[i0:i1] = Xc
        y[i0:i1] = np.cos(4.0 * Xc).sum(axis=1) + 0.1 * rng.standard_normal(i1 - i0)
    Xt = rng.random((m, d)).astype(np.float32)
    return Problem(name="taxi", X=X, Y=y[:, None], Xtest=Xt, kernel=RBF, ell=0.5,
                   sigma2=1.0, lam=1e-2, b=b if b is not None else min(100000, n // 4),
                   r=100, iters=None)


def injected_schedule(n, b, r, T, seed=1234):
    """Host-drawn randomness for parity runs: arrays B (T,b) int64, Omega (T,b,r), v0 (T,b).

    B rows are distinct uniform indices; Omega has N(0, 1/b) entries; v0 ~ N(0, I).
    Both the CUDA path and the oracle consume exactly these values.
    """
    rng = np.random.default_rng(seed)
    B = np.stack([rng.choice(n, size=b, replace=False) for _ in range(T)]).astype(np.int64)
    Om = (rng.standard_normal((T, b, r)) / np.sqrt(b)).astype(np.float32)
    v0 = rng.standard_normal((T, b)).astype(np.float32)
    return B, Om, v0


def schedule_fn(B, Om, v0):
    """Wrap injected arrays as a schedule t -> (B_t, Omega_t, v0_t) in float64."""
    def sched(t):
        return B[t], Om[t].astype(np.float64), v0[t].astype(np.float64)
    return sched


def rf_draws(q, d, dof, ns, n, noise, seed=7):
    """Randomness of the random-feature prior and of pathwise conditioning:
    z (q, d) ~ N(0, 1), u (q,) ~ chi^2(dof) (None when dof is None), phase (q,) ~ U[0, 2 pi),
    theta (q, ns) ~ N(0, 1), zeta (n, ns) ~ N(0, noise).  All float32."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((q, d)).astype(np.float32)
    u = rng.chisquare(dof, q).astype(np.float32) if dof is not None else None
    phase = rng.uniform(0.0, 2.0 * np.pi, q).astype(np.float32)
    theta = rng.standard_normal((q, ns)).astype(np.float32)
    zeta = (np.sqrt(noise) * rng.standard_normal((n, ns))).astype(np.float32)
    return z, u, phase, theta, zeta
