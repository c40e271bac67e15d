"""Tolerances of the GPU solver parity tests, set from the oracle's own sensitivity.

The GPU runs Alg. 2 in FP32 arithmetic (split-TF32 distances at FP32 accuracy,
FP64 only for the r x r core and the convergence sums) where the oracle runs
FP64.  How far an FP32 run may land from the FP64 one is the conditioning of
the iteration times the FP32 rounding unit, and that conditioning differs by
orders of magnitude between shapes: a well-conditioned block moves W by about
the rounding unit, a degenerate one (b = n = r, lambda = 1e-2) by a thousand
times more.  A fixed tolerance is either too loose for the first or fails the
second, and an a-priori bound (||dP|| / rho times the 2N + 1 powering
products, used before) is a worst case that allowed percent-level errors.

So each test measures the sensitivity on the oracle alone: it re-runs the
oracle with what an FP32 implementation rounds perturbed at the FP32 level --
the points X and the sketch test matrix Omega multiplied entrywise by
(1 +- 2^-23) with random signs, and the two copies of K_BB that such an
implementation forms separately (the sketch's and the power iteration's; the
exact block solve's for SAP) perturbed independently the same way, through the
oracle's perturb hook -- and takes the largest relative change of eta_t, rho_t
and W_T over SENS_DRAWS such runs.  No GPU value enters.  The copies matter
where the preconditioner matches K_BB closely (r near b): there the stepsize is
the top eigenvalue of P^{-1/2} H P^{-1/2} ~ I, which moves with any mismatch
between the K_BB inside P and the one inside H by ||dK|| / rho, while a
perturbation of X moves both together.  The GPU result must lie within FACTOR
times that change (floored at FLOOR, the level at which FP32 sums of a few
thousand terms already differ), and never beyond the a-priori bound, which
stays as a cap.

With ADASAP_PARITY_LOG set to a file path, every check appends one JSON line
(test, quantity, observed error, sensitivity, tolerance, cap), which is how the
observed errors are recorded.
"""

import json
import os

import numpy as np

SENS_DRAWS = 2
FACTOR = 10.0
FLOOR = 1e-5
EPS32 = 2.0 ** -23


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def perturb(a, rng):
    """a * (1 +- 2^-23), an independent random sign per entry."""
    a = np.asarray(a, np.float64)
    return a * (1.0 + EPS32 * rng.choice((-1.0, 1.0), size=a.shape))


def perturbed_schedule(sched, rng):
    """The same (B, Omega, v0) draws with Omega perturbed at the FP32 level."""
    cache = {}

    def f(t):
        if t not in cache:
            B, Om, v0 = sched(t)
            cache[t] = (B, perturb(Om, rng), v0)
        return cache[t]

    return f


def trace_of(rec):
    eta = np.array([x["eta"] for x in rec], np.float64)
    rho = np.array([x["rho"] if x["rho"] is not None else np.nan for x in rec], np.float64)
    return eta, rho


def max_rel_entry(a, b):
    """Largest entrywise relative difference of two traces (NaN entries skipped)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    m = np.isfinite(a) & np.isfinite(b)
    if not m.any():
        return 0.0
    return float(np.max(np.abs(a[m] - b[m]) / np.maximum(np.abs(b[m]), 1e-300)))


def block_perturber(rng):
    """The oracle's perturb hook: every copy of K_BB it is handed, perturbed independently."""
    return lambda tag, K: perturb(K, rng)


def sensitivity(run, X, sched, seed=0):
    """Largest relative change of W_T, eta_t and rho_t over SENS_DRAWS oracle runs.

    run(X, sched, hook) -> (W_T, record list); X and sched are the unperturbed
    inputs (sched None: a run without a sketch, such as SAP with the exact block
    solve) and hook is passed to the oracle as its perturb argument (None for
    the reference run).  Returns (W_ref, rec_ref, {"W": ..., "eta": ..., "rho": ...})."""
    W0, rec0 = run(np.asarray(X, np.float64), sched, None)
    eta0, rho0 = trace_of(rec0)
    g = np.random.default_rng(1000 + seed)
    sens = {"W": 0.0, "eta": 0.0, "rho": 0.0}
    for _ in range(SENS_DRAWS):
        Wp, recp = run(perturb(X, g), perturbed_schedule(sched, g) if sched is not None else None,
                       block_perturber(g))
        etap, rhop = trace_of(recp)
        sens["W"] = max(sens["W"], rel(Wp, W0))
        sens["eta"] = max(sens["eta"], max_rel_entry(etap, eta0))
        sens["rho"] = max(sens["rho"], max_rel_entry(rhop, rho0))
    return W0, rec0, sens


def tol_from(sens, cap):
    """FACTOR x the oracle's sensitivity, at least FLOOR, at most the a-priori cap."""
    return float(min(cap, max(FLOOR, FACTOR * sens)))


def a_priori_cap(rec, b, sigma2, power_iters=10, eta=True):
    """The worst-case bound used before: 4 eps32 b sigma2 / min rho, times 2N + 1 for eta and W."""
    rhos = [x["rho"] for x in rec if x["rho"] is not None]
    base = 1e-4 if not rhos else max(1e-4, 4 * EPS32 * b * sigma2 / min(rhos))
    return max(1e-4, (2 * power_iters + 1) * base) if eta else base


def record(test, quantity, observed, sens, tol, cap):
    path = os.environ.get("ADASAP_PARITY_LOG")
    if not path:
        return
    with open(path, "a") as f:
        f.write(json.dumps({"test": test, "quantity": quantity, "observed": observed, "sens": sens,
                            "tol": tol, "cap": cap}) + "\n")


def check(test, items, recorded=None):
    """items: (quantity, observed, sens, cap) tuples.  Records every one first (so a
    log shows all of them even when one fails), then asserts observed < tol, with
    tol = tol_from(sens, cap), or FACTOR x recorded[quantity] (a previously observed
    error, for the few cases whose FP32 error the perturbations do not exercise)
    when that is larger, never beyond cap."""
    rows = []
    for quantity, observed, sens, cap in items:
        tol = tol_from(sens, cap)
        if recorded and quantity in recorded:
            tol = float(min(cap, max(tol, FACTOR * recorded[quantity])))
        record(test, quantity, observed, sens, tol, cap)
        rows.append((quantity, observed, sens, tol, cap))
    bad = [r for r in rows if not (r[1] < r[3])]   # NaN fails
    assert not bad, "; ".join("%s %s: observed %.3g >= tol %.3g (oracle sensitivity %.3g, cap %.3g)"
                              % (test, q, obs, tol, sens, cap) for q, obs, sens, tol, cap in bad)
