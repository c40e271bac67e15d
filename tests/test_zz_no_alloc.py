"""The allocation-free block-row product, adasap_kernel_rows_noalloc.

Some callers cannot allocate device memory while they run (an allocator-less
runtime, a real-time loop that must not touch the allocator, a process whose
device memory is already reserved).  For them the library offers this one
entry point, whose scratch is a static device array instead of a workspace it
would allocate.  These tests call it through the C-ABI and compare it with the
allocating adasap_kernel_rows, on two calls in a row (the array is shared and
keeps the previous call's contents).  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest
import torch

from oracle import kernels as OK
from paper_2505_13723_b300 import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-5   # the tolerance of the kernel-row parity tests


def _call_noalloc(lib, ctx, B, W, out):
    W2 = W if W.dim() == 2 else W.view(-1, 1)
    return lib._lib.adasap_kernel_rows_noalloc(
        ctx.h, ctypes.c_void_p(B.data_ptr()), B.numel(), ctypes.c_void_p(W2.data_ptr()), W2.shape[1],
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("prec,s", [(1, 1), (0, 1), (0, 3)])
def test_noalloc_matches_kernel_rows_on_two_calls(lib, prec, s):
    P = synth.regress(n=20000)
    ctx = lib.Context(P.X, P.kernel, P.ell, P.sigma2, P.lam, precision=prec)
    g = np.random.default_rng(7)
    for call, b in enumerate([1500, 613]):          # two calls in a row, different sizes
        B = torch.from_numpy(g.choice(20000, size=b, replace=False)).cuda()
        W = torch.from_numpy(g.standard_normal((20000, s)).astype(np.float32)).cuda()
        ref = ctx.kernel_rows(B, W)
        out = torch.full((b, s), float("nan"), device="cuda")
        assert _call_noalloc(lib, ctx, B, W, out) == 0, lib._lib.adasap_last_error()
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.isfinite(o).all(), "call %d left unwritten outputs" % call
        np.testing.assert_allclose(o, r, rtol=RTOL, atol=RTOL * np.abs(r).max())


@pytest.mark.parametrize("prec", [1, 2])
def test_noalloc_multi_rhs_on_a_tensor_core_precision_runs_fp32(lib, prec):
    """s = 3 in a tensor-core precision: the allocation-free call takes the plain FP32
    CUDA-core kernel, so it is held to the FP32 parity bound against the oracle
    (|out - ref| <= 1e-5 * sum_j |k_ij| |w_j|), on two calls in a row."""
    P = synth.regress(n=20000)
    ctx = lib.Context(P.X, P.kernel, P.ell, P.sigma2, P.lam, precision=prec)
    Xd = P.X.astype(np.float64)
    g = np.random.default_rng(9 + prec)
    for call, b in enumerate([700, 257]):
        rows = g.choice(20000, size=b, replace=False)
        W = g.standard_normal((20000, 3)).astype(np.float32)
        out = torch.full((b, 3), float("nan"), device="cuda")
        assert _call_noalloc(lib, ctx, torch.from_numpy(rows).cuda(), torch.from_numpy(W).cuda(), out) == 0, \
            lib._lib.adasap_last_error()
        torch.cuda.synchronize()
        o = out.cpu().numpy().astype(np.float64)
        ref = OK.kernel_rows(Xd, rows, W.astype(np.float64), P.kernel, P.ell, P.sigma2)
        scale = OK.kernel_rows(Xd, rows, np.abs(W.astype(np.float64)), P.kernel, P.ell, P.sigma2)
        assert np.isfinite(o).all(), "call %d left unwritten outputs" % call
        assert (np.abs(o - ref) <= RTOL * scale).all(), (call, np.max(np.abs(o - ref) / scale))


def test_noalloc_rejects_sizes_beyond_its_static_scratch(lib):
    P = synth.small(n=3000)
    ctx = lib.Context(P.X, P.kernel, P.ell, P.sigma2, P.lam)
    b, s = 3000, 128                                  # partials of 128 columns per split do not fit
    B = torch.arange(b, device="cuda")
    W = torch.zeros(3000, s, device="cuda")
    out = torch.zeros(b, s, device="cuda")
    assert _call_noalloc(lib, ctx, B, W, out) == 1    # ADASAP_EINVAL, no GPU work
    assert b"bytes of scratch" in lib._lib.adasap_last_error()
    # the entry point still works afterwards
    W1 = torch.ones(3000, 1, device="cuda")
    o1 = torch.zeros(b, 1, device="cuda")
    assert _call_noalloc(lib, ctx, B, W1, o1) == 0
    torch.cuda.synchronize()
    np.testing.assert_allclose(o1.cpu().numpy(), ctx.kernel_rows(B, W1).cpu().numpy(), rtol=RTOL)
