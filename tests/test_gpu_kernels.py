"""GPU parity of the kernel-row engine, sampler, posterior mean and adjoint
against the FP64 oracle (through the C-ABI)."""

import numpy as np
import pytest
import torch

from oracle import gp
from oracle import kernels as OK
from oracle import rng as OR
from paper_2505_13723_b300 import synth

pytestmark = pytest.mark.gpu

# Tolerance of an FP32 kernel-row product (the stated bound: <= 1e-5 relative):
#   |out_i - ref_i| <= 1e-5 * sum_j |k_ij| |w_ij|
# i.e. relative to the sum of absolute terms, the scale at which FP32
# rounding of distances, exponentials and partial sums acts.
RTOL_ROWS = 1e-5


def _data(n, d, s, seed, dist="normal"):
    g = np.random.default_rng(seed)
    X = (g.standard_normal((n, d)) if dist == "normal" else g.random((n, d))).astype(np.float32)
    W = g.standard_normal((n, s)).astype(np.float32)
    return X, W


def _check_rows(got, X, rows, W, kern, ell, s2, rtol=RTOL_ROWS):
    Xd = X.astype(np.float64)
    ref = OK.kernel_apply(Xd[rows], Xd, W.astype(np.float64), kern, ell, s2)
    scale = OK.kernel_apply(Xd[rows], Xd, np.abs(W.astype(np.float64)), kern, ell, s2)
    err = np.abs(got - ref)
    bad = ~(err <= rtol * scale + 1e-30)     # NaN outputs fail too
    assert not bad.any(), "max err/scale %.3e" % (err / np.maximum(scale, 1e-300)).max()


def _ctx(lib, X, kern, ell, s2, lam, prec):
    ctx = lib.Context(X, kern, ell, s2, lam)
    if prec == lib.PREC_TF32X3 and X.shape[1] + 2 > 32:
        pytest.skip("tensor-core path needs d <= 30")
    ctx.set_precision(prec)
    return ctx


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kern", [0, 1, 2])
@pytest.mark.parametrize("d", [1, 8, 11, 20, 40])
@pytest.mark.parametrize("s", [1, 3, 4, 17, 64])
def test_kernel_rows_matches_oracle(lib, kern, d, s, prec):
    n, b = 3001, 157                      # ragged against every tile size
    X, W = _data(n, d, s, seed=d * 10 + s)
    ell = 0.9 * np.sqrt(d)
    ctx = _ctx(lib, X, kern, ell, 1.3, 1e-2, prec)
    g = np.random.default_rng(kern)
    rows = g.choice(n, size=b, replace=False)
    out = ctx.kernel_rows(torch.from_numpy(rows).cuda(), torch.from_numpy(W).cuda()).cpu().numpy()
    _check_rows(out.astype(np.float64), X, rows, W, kern, ell, 1.3)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("s", [1, 100])
def test_kernel_rows_edge_sizes(lib, s, prec):
    # n = 1, b = 1; a block of all rows; repeated rows
    X, W = _data(1, 3, s, seed=1)
    ctx = _ctx(lib, X, 1, 1.0, 1.0, 1.0, prec)
    out = ctx.kernel_rows(torch.zeros(1, dtype=torch.int64, device="cuda"), torch.from_numpy(W).cuda())
    np.testing.assert_allclose(out.cpu().numpy(), W, rtol=1e-6)      # k(x, x) = sigma2 = 1
    X, W = _data(700, 5, s, seed=2)
    ctx = _ctx(lib, X, 2, 1.5, 0.7, 1.0, prec)
    rows = np.concatenate([np.arange(700), [3, 3, 699]])
    out = ctx.kernel_rows(torch.from_numpy(rows).cuda(), torch.from_numpy(W).cuda()).cpu().numpy()
    _check_rows(out.astype(np.float64), X, rows, W, 2, 1.5, 0.7)


@pytest.mark.parametrize("s,kern,d", [(2, 0, 3), (128, 1, 16), (33, 2, 9), (100, 1, 11)])
def test_multi_rhs_tensor_core_product_spans_splits(lib, s, kern, d):
    """s >= 2 on the tensor cores (kernel tile x W contraction in TMEM): more columns
    than one accumulator span (several column splits), a ragged last tile, s up to 128."""
    n, b = 40077, 300
    X, W = _data(n, d, s, seed=s + kern)
    ell = 0.8 * np.sqrt(d)
    ctx = _ctx(lib, X, kern, ell, 0.9, 1e-2, lib.PREC_TF32X3)
    rows = np.random.default_rng(s).choice(n, size=b, replace=False)
    out = ctx.kernel_rows(torch.from_numpy(rows).cuda(), torch.from_numpy(W).cuda()).cpu().numpy()
    _check_rows(out.astype(np.float64), X, rows, W, kern, ell, 0.9)


@pytest.mark.parametrize("kern,d,s", [(0, 16, 64), (1, 11, 2), (2, 8, 100)])
def test_multi_rhs_single_pass_tf32_contraction(lib, kern, d, s):
    """ADASAP_PREC_TF32: one MMA on TF32-rounded kernel values and W (2^-11 relative
    rounding each, so a product is off by at most ~2^-10 relative, plus the FP32
    accumulation): held to 3e-3 of sum_j |k_ij||w_j|, the low-precision bound; the
    typical error is far inside it and still far above the split form's."""
    n, b = 20011, 257
    X, W = _data(n, d, s, seed=3 * s + kern)
    ell = 0.8 * np.sqrt(d)
    ctx = _ctx(lib, X, kern, ell, 1.1, 1e-2, lib.PREC_TF32)
    rows = np.random.default_rng(s).choice(n, size=b, replace=False)
    out = ctx.kernel_rows(torch.from_numpy(rows).cuda(), torch.from_numpy(W).cuda()).cpu().numpy()
    _check_rows(out.astype(np.float64), X, rows, W, kern, ell, 1.1, rtol=3e-3)
    Xd = X.astype(np.float64)
    ref = OK.kernel_apply(Xd[rows], Xd, W.astype(np.float64), kern, ell, 1.1)
    scale = OK.kernel_apply(Xd[rows], Xd, np.abs(W.astype(np.float64)), kern, ell, 1.1)
    assert np.median(np.abs(out - ref) / scale) < 3e-4


@pytest.mark.parametrize("s", [5, 17])
def test_fp32_wide_product_with_empty_column_splits(lib, s):
    """n = 40,077 columns over the CUDA-core split count leaves the last splits without
    columns; their partial sums must still be written (as zeros)."""
    n, b = 40077, 300
    X, W = _data(n, 11, s, seed=11 + s, dist="uniform")
    ctx = _ctx(lib, X, 0, 0.3, 1.0, 1e-3, lib.PREC_FP32)
    rows = np.arange(b)
    for _ in range(2):
        out = ctx.kernel_rows(torch.from_numpy(rows).cuda(), torch.from_numpy(W).cuda()).cpu().numpy()
        _check_rows(out.astype(np.float64), X, rows, W, 0, 0.3, 1.0)


@pytest.mark.parametrize("kern", [0, 1])
def test_multi_rhs_tensor_core_product_many_items_per_cta(lib, kern):
    """All 10,000 rows against 10,000 columns with s = 100 (the sketch K_BB Omega of
    the 1M-point workload): more (row tile, split) items than CTAs, so every CTA
    carries its pipeline phases across items; sampled rows against the oracle."""
    n, d, s = 10000, 11, 100
    X, W = _data(n, d, s, seed=7, dist="uniform")
    ctx = _ctx(lib, X, kern, 0.3, 1.0, 1e-3, lib.PREC_TF32X3)
    rows = np.arange(n)
    out = ctx.kernel_rows(torch.from_numpy(rows).cuda(), torch.from_numpy(W).cuda()).cpu().numpy()
    pick = np.random.default_rng(kern).choice(n, size=200, replace=False)
    pick = np.concatenate([pick, [0, 127, 128, n - 1]])
    _check_rows(out[pick].astype(np.float64), X, pick, W, kern, 0.3, 1.0)


@pytest.mark.parametrize("m,n,kern", [(4999, 20011, 1), (2500, 50001, 2), (9999, 10001, 0)])
def test_tensor_core_flat_schedule_ragged(lib, m, n, kern):
    """Single-RHS tensor-core products whose tiles are cut into equal runs per CTA
    (the flat schedule: at these sizes a row tile meets up to 5, 9 and 3 CTAs, each
    writing its own partial slot and the last one zeroing the rest), with the last
    row tile and the last column tile ragged.  Rows sampled from every row tile,
    plus the whole last one."""
    d = 11
    X, W = _data(n, d, 1, seed=m + kern)
    ell = 0.8 * np.sqrt(d)
    ctx = _ctx(lib, X, kern, ell, 0.7, 1e-3, lib.PREC_TF32X3)
    g = np.random.default_rng(m)
    rows = g.choice(n, size=m, replace=False)
    out = ctx.kernel_rows(torch.from_numpy(rows).cuda(), torch.from_numpy(W).cuda()).cpu().numpy()
    last = (m - 1) // 128 * 128
    pick = np.unique(np.concatenate([g.choice(last, size=300, replace=False), np.arange(last, m)]))
    _check_rows(out[pick].astype(np.float64), X, rows[pick], W, kern, ell, 0.7)


@pytest.mark.parametrize("prec,s", [(0, 2), (1, 1), (1, 2)])
def test_kernel_rows_invalid_index_gives_nan_row(lib, prec, s):
    X, W = _data(500, 4, s, seed=3)
    ctx = _ctx(lib, X, 0, 1.0, 1.0, 1.0, prec)
    rows = torch.tensor([0, -1, 499, 500, 7], device="cuda")
    out = ctx.kernel_rows(rows, torch.from_numpy(W).cuda()).cpu().numpy()
    assert np.isnan(out[1]).all() and np.isnan(out[3]).all()
    assert np.isfinite(out[[0, 2, 4]]).all()
    _check_rows(out[[0, 2, 4]].astype(np.float64), X, np.array([0, 499, 7]), W, 0, 1.0, 1.0)


@pytest.mark.parametrize("prec", [0, 1])
def test_kernel_rows_regress_workload_full_size_sampled(lib, prec):
    """n = 2^20, d = 11, Matern-3/2, b = 10^4 (the benchmark's launch); 48 rows checked."""
    P = synth.regress()
    ctx = _ctx(lib, P.X, P.kernel, P.ell, P.sigma2, P.lam, prec)
    g = np.random.default_rng(11)
    rows = g.choice(P.X.shape[0], size=P.b, replace=False)
    W = g.standard_normal((P.X.shape[0], 1)).astype(np.float32)
    out = ctx.kernel_rows(torch.from_numpy(rows).cuda(), torch.from_numpy(W).cuda()).cpu().numpy()
    pick = g.choice(P.b, size=48, replace=False)
    _check_rows(out[pick].astype(np.float64), P.X, rows[pick], W, P.kernel, P.ell, P.sigma2)


@pytest.mark.parametrize("prec", [1, 2])
def test_kernel_rows_multirhs_workload_full_size_sampled(lib, prec):
    """n = 2^18, d = 16, RBF, b = 4096, s = 64 (the multi-RHS Step I launch the benchmark
    times); 24 rows checked, at the split (1e-5) and single-pass TF32 (3e-3) bounds."""
    P = synth.multirhs()
    ctx = _ctx(lib, P.X, P.kernel, P.ell, P.sigma2, P.lam, prec)
    g = np.random.default_rng(12)
    rows = g.choice(P.X.shape[0], size=P.b, replace=False)
    out = ctx.kernel_rows(torch.from_numpy(rows).cuda(), torch.from_numpy(P.Y).cuda()).cpu().numpy()
    pick = g.choice(P.b, size=24, replace=False)
    _check_rows(out[pick].astype(np.float64), P.X, rows[pick], P.Y, P.kernel, P.ell, P.sigma2,
                rtol=RTOL_ROWS if prec == 1 else 3e-3)


def test_kernel_rows_unaligned_rhs_view(lib):
    """A contiguous W that starts 4 bytes past an allocation (no 16-byte alignment)."""
    X, W = _data(900, 6, 1, seed=12)
    ctx = lib.Context(X, 1, 1.2, 1.0, 1e-2)
    buf = torch.zeros(901, device="cuda")
    buf[1:] = torch.from_numpy(W[:, 0]).cuda()
    rows = np.arange(0, 900, 3)
    out = ctx.kernel_rows(torch.from_numpy(rows).cuda(), buf[1:]).cpu().numpy()
    _check_rows(out.astype(np.float64), X, rows, W, 1, 1.2, 1.0)


def test_sampler_matches_oracle_generator(lib):
    for (n, b, r, t, seed) in [(2000, 200, 32, 0, 0), (2000, 200, 32, 7, 0), (1 << 20, 10000, 100, 3, 99),
                               (5, 5, 2, 1, 1), (1, 1, 1, 0, 2)]:
        B, Om, v0 = lib.sample(seed, t, n, b, r)
        np.testing.assert_array_equal(B.cpu().numpy(), OR.sample_block(n, b, seed, t))
        np.testing.assert_allclose(Om.cpu().numpy(), OR.sample_omega(b, r, seed, t), rtol=2e-5, atol=2e-6)
        np.testing.assert_allclose(v0.cpu().numpy(), OR.sample_v0(b, seed, t), rtol=2e-5, atol=2e-6)


@pytest.mark.parametrize("prec,s", [(0, 2), (1, 1)])
@pytest.mark.parametrize("kern", [0, 1, 2])
def test_predict_matches_oracle(lib, kern, prec, s):
    X, W = _data(2500, 6, s, seed=5)
    Xt = np.random.default_rng(6).standard_normal((333, 6)).astype(np.float32)
    ctx = _ctx(lib, X, kern, 1.1, 0.8, 1e-2, prec)
    out = ctx.predict(torch.from_numpy(Xt).cuda(), torch.from_numpy(W).cuda()).cpu().numpy()
    ref = gp.posterior_mean(Xt.astype(np.float64), X.astype(np.float64), W.astype(np.float64), kern, 1.1, 0.8)
    scale = gp.posterior_mean(Xt.astype(np.float64), X.astype(np.float64), np.abs(W.astype(np.float64)), kern, 1.1, 0.8)
    assert (np.abs(out - ref) <= RTOL_ROWS * scale).all()


@pytest.mark.parametrize("kern", [0, 1, 2])
@pytest.mark.parametrize("s", [1, 3])
def test_hypergrad_matches_oracle(lib, kern, s):
    X, W = _data(1500, 5, s, seed=7)
    G = np.random.default_rng(8).standard_normal(W.shape).astype(np.float32)
    ctx = lib.Context(X, kern, 0.9, 1.4, 1e-2)
    d_ell, d_s2 = ctx.hypergrad(torch.from_numpy(W).cuda(), torch.from_numpy(G).cuda())
    r_ell, r_s2 = gp.hypergrad(X.astype(np.float64), W.astype(np.float64), G.astype(np.float64), kern, 0.9, 1.4)
    # scale: the same sums with absolute values (cancellation-aware bound)
    Xd = X.astype(np.float64)
    a_ell = np.sum(np.abs(G) * OK.kernel_apply(Xd, Xd, np.abs(W.astype(np.float64)), kern, 0.9, 1.4, deriv=True))
    a_s2 = np.sum(np.abs(G) * OK.kernel_apply(Xd, Xd, np.abs(W.astype(np.float64)), kern, 0.9, 1.4)) / 1.4
    assert abs(d_ell - r_ell) <= 1e-5 * a_ell
    assert abs(d_s2 - r_s2) <= 1e-5 * a_s2


def test_hypergrad_at_16384_against_finite_differences(lib):
    """The adjoint at n = 16,384 (BO-shaped data, Matern-5/2) against central differences of
    the kernel-row product itself: f(theta) = sum G * (K(theta) W)."""
    P = synth.bo_systems(count=1)[0]
    g = np.random.default_rng(9)
    n = 16384
    X = g.uniform(-1, 1, (n, 8)).astype(np.float32)
    W = g.standard_normal((n, 1)).astype(np.float32)
    G = g.standard_normal((n, 1)).astype(np.float32)
    ell, s2 = 0.6, 1.0
    Wt, Gt = torch.from_numpy(W).cuda(), torch.from_numpy(G).cuda()
    rows = torch.arange(n, device="cuda")

    def f(e, s):
        c = lib.Context(X, P.kernel, e, s, 1e-3)
        return float((c.kernel_rows(rows, Wt).double() * Gt.double()).sum())

    ctx = lib.Context(X, P.kernel, ell, s2, 1e-3)
    d_ell, d_s2 = ctx.hypergrad(Wt, Gt)
    h = 1e-2 * ell
    fd_ell = (f(ell + h, s2) - f(ell - h, s2)) / (2 * h)
    fd_s2 = (f(ell, s2 + 0.1) - f(ell, s2 - 0.1)) / 0.2
    assert abs(d_ell - fd_ell) <= 2e-3 * abs(fd_ell)
    assert abs(d_s2 - fd_s2) <= 1e-4 * abs(fd_s2)


def test_hypergrad_at_16384_against_oracle_on_sampled_rows(lib):
    """The adjoint at n = 16,384 (BO-shaped data, Matern-5/2, s = 2) against the oracle's
    hypergradient: G is non-zero on 300 sampled rows only, so the oracle's sums
    sum_i G_i (dK/dell W)_i and sum_i G_i (K W)_i / sigma2 need those 300 kernel rows,
    while the GPU's adjoint still runs over all n x n entries (the zero rows add
    nothing).  Held to 1e-5 of the same sums with absolute values."""
    g = np.random.default_rng(19)
    n, d, s = 16384, 8, 2
    X = g.uniform(-1, 1, (n, d)).astype(np.float32)
    W = g.standard_normal((n, s)).astype(np.float32)
    G = np.zeros((n, s), np.float32)
    rows = np.sort(g.choice(n, size=300, replace=False))
    G[rows] = g.standard_normal((300, s))
    ell, s2, kern = 0.6, 1.3, 2
    ctx = lib.Context(X, kern, ell, s2, 1e-3)
    d_ell, d_s2 = ctx.hypergrad(torch.from_numpy(W).cuda(), torch.from_numpy(G).cuda())
    Xd, Wd, Gd = X.astype(np.float64), W.astype(np.float64), G[rows].astype(np.float64)
    dKW = OK.kernel_apply(Xd[rows], Xd, Wd, kern, ell, s2, deriv=True)
    KW = OK.kernel_apply(Xd[rows], Xd, Wd, kern, ell, s2)
    r_ell, r_s2 = float(np.sum(Gd * dKW)), float(np.sum(Gd * KW) / s2)
    a_ell = float(np.sum(np.abs(Gd) * OK.kernel_apply(Xd[rows], Xd, np.abs(Wd), kern, ell, s2, deriv=True)))
    a_s2 = float(np.sum(np.abs(Gd) * OK.kernel_apply(Xd[rows], Xd, np.abs(Wd), kern, ell, s2)) / s2)
    assert abs(d_ell - r_ell) <= 1e-5 * a_ell, (d_ell, r_ell, a_ell)
    assert abs(d_s2 - r_s2) <= 1e-5 * a_s2, (d_s2, r_s2, a_s2)


def test_autograd_function_gradients(lib):
    X, W = _data(800, 4, 2, seed=10)
    ctx = lib.Context(X, 1, 0.7, 1.2, 1e-2)
    Wt = torch.from_numpy(W).cuda().requires_grad_(True)
    ell = torch.tensor(0.7, device="cuda", requires_grad=True)
    s2 = torch.tensor(1.2, device="cuda", requires_grad=True)
    G = torch.randn(800, 2, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    y = lib.KernelMatmul.apply(ctx, Wt, ell, s2)
    (y * G).sum().backward()
    Xd = X.astype(np.float64)
    Kd = OK.kernel_matrix(Xd, Xd, 1, 0.7, 1.2)
    np.testing.assert_allclose(y.detach().cpu().numpy(), Kd @ W, rtol=0, atol=1e-5 * (np.abs(Kd) @ np.abs(W)).max())
    Gn = G.cpu().numpy().astype(np.float64)
    gW_ref = Kd @ Gn
    assert np.abs(Wt.grad.cpu().numpy() - gW_ref).max() <= 1e-5 * (np.abs(Kd) @ np.abs(Gn)).max()
    r_ell, r_s2 = gp.hypergrad(Xd, W.astype(np.float64), Gn, 1, 0.7, 1.2)
    assert abs(ell.grad.item() - r_ell) <= 1e-4 * abs(r_ell) + 1e-3
    assert abs(s2.grad.item() - r_s2) <= 1e-4 * abs(r_s2) + 1e-3


def test_fma_pipe_sqrt_is_correctly_rounded_on_a_dense_grid(lib):
    """The square root the Matern epilogues take on the FMA pipe (Newton steps from a
    bit-pattern seed): within half an ulp of the correctly rounded square root on
    2^22 points spread log-uniformly over [1e-30, 1e21] plus every float in [1, 4)
    spaced 64 ulps apart, exactly 0 -> 1e-15 (the documented clamp), and no worse
    than the special-function unit's sqrt.approx on the same points."""
    g = np.random.default_rng(21)
    x = np.exp(g.uniform(np.log(1e-30), np.log(1e21), 1 << 22)).astype(np.float32)
    dense = np.arange(np.float32(1.0).view(np.int32), np.float32(4.0).view(np.int32), 64,
                      dtype=np.int32).view(np.float32)
    x = np.concatenate([x, dense])
    xt = torch.from_numpy(x).cuda()
    got = lib.eval_math(0, xt).cpu().numpy().astype(np.float64)
    mufu = lib.eval_math(1, xt).cpu().numpy().astype(np.float64)
    exact = np.sqrt(x.astype(np.float64))
    ulp = np.spacing(exact.astype(np.float32)).astype(np.float64)
    err = np.abs(got - exact) / ulp
    assert err.max() <= 0.5 + 1e-3, err.max()
    assert err.max() <= (np.abs(mufu - exact) / ulp).max() + 1e-3
    z = lib.eval_math(0, torch.zeros(4, device="cuda")).cpu().numpy()
    np.testing.assert_allclose(z, 1e-15, rtol=1e-6)
