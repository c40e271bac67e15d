"""FP64 CPU oracle for the ADASAP hot path -- TEST INFRASTRUCTURE ONLY.

This package restates, in plain NumPy/SciPy at float64, what the paper
"Turbocharging Gaussian Process Inference with Approximate Sketch-and-Project"
(Rathore, Frangella, Garg, Derezinski, Udell, NeurIPS 2025) computes on its hot
path.  It exists so that the CUDA path can be checked against something that a
reader can compare with the paper by eye.  Only ``tests/``, the package entry
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product path never calls it and shares
no code with it (the seeded input generators in ``paper_2505_13723_b300.synth``
are the one module both sides read, and that module holds none of the method's
arithmetic).

Modules
-------
kernels  -- RBF / Matern-3/2 / Matern-5/2 kernels, their lengthscale
            derivatives, brute-force kernel-row products (Sec. 2, eq. post_eqns).
rng      -- Philox4x32-10 counter-based generator, the keyed Feistel
            permutation used to draw b distinct rows, Box-Muller normals.
adasap   -- Alg. 1 (SAP), Alg. 2 (ADASAP), Alg. 4 (Nystrom), the Woodbury
            applies of App. C.2, Alg. 5 (GetStepsize), Alg. 6 (NesterovAcc).
gp       -- dense Cholesky reference solve, posterior mean, residuals,
            hyperparameter adjoint.
pathwise -- random-feature prior draws, pathwise-conditioned posterior
            samples (Sec. 2.1), the textbook posterior covariance, test RMSE
            and NLL.

Parity status: every public function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against something other than itself (a library
routine, a closed form, a published known-answer vector, brute force, or an
exact special case).  No function here is "parity unpinned".
"""

from . import kernels, rng, adasap, gp  # noqa: F401
