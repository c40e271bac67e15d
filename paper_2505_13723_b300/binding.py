"""Thin ctypes binding over the C-ABI in include/adasap.h.

Argument marshalling only: every step of the ADASAP path runs in the CUDA
library.  Device buffers and streams come from PyTorch.  Importing this module
loads _lib/libadasap.so and raises ImportError if it has not been built
(``python -m paper_2505_13723_b300.build``); there is no CPU fallback.
"""

import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libadasap.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("CUDA library %s is missing: run `python -m paper_2505_13723_b300.build`" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)

RBF, MATERN32, MATERN52 = 0, 1, 2
PREC_FP32, PREC_TF32X3, PREC_TF32 = 0, 1, 2
KERNELS = {"rbf": RBF, "matern32": MATERN32, "matern52": MATERN52}

STATUS = {0: "ADASAP_OK", 1: "ADASAP_EINVAL", 2: "ADASAP_ENOMEM", 3: "ADASAP_ECUDA",
          4: "ADASAP_ENUMERIC", 5: "ADASAP_EDIVERGED", 6: "ADASAP_ETIMEOUT",
          7: "ADASAP_ENOTCONVERGED"}

# exported symbols, kept in step with include/adasap.h (a CPU test checks both)
SYMBOLS = ["adasap_default_opts", "adasap_status_string", "adasap_last_error", "adasap_create",
           "adasap_destroy", "adasap_kernel_rows", "adasap_solve", "adasap_solve_scheduled",
           "adasap_predict", "adasap_hypergrad", "adasap_sample", "adasap_solver_begin",
           "adasap_solver_step", "adasap_solver_residual", "adasap_solver_get_w",
           "adasap_solver_scalars", "adasap_solver_end", "adasap_solver_graph_kernels",
           "adasap_solver_diag", "adasap_set_precision",
           "adasap_kernel_rows_noalloc", "adasap_measure_pipes", "adasap_residual",
           "adasap_solve_batched", "adasap_rf_prior", "adasap_pathwise", "adasap_rmse_nll",
           "adasap_check_device", "adasap_wait_selftest", "adasap_solver_get_state",
           "adasap_solver_set_state", "adasap_schedule_check", "adasap_eval_math"]


class Opts(ctypes.Structure):
    _fields_ = [("b", ctypes.c_int64), ("r", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("tol", ctypes.c_double), ("power_iters", ctypes.c_int), ("mu", ctypes.c_double),
                ("nu", ctypes.c_double), ("precond", ctypes.c_int), ("literal", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("check_every", ctypes.c_int),
                ("check_rows", ctypes.c_int64), ("eps", ctypes.c_double), ("tail_average", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_resid", ctypes.c_double),
                ("resid_exact", ctypes.c_int), ("seconds", ctypes.c_double),
                ("last_eta", ctypes.c_double), ("last_rho", ctypes.c_double),
                ("status_detail", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_lib.adasap_default_opts.argtypes = [ctypes.POINTER(Opts), _I64]
_lib.adasap_default_opts.restype = None
_lib.adasap_status_string.argtypes = [ctypes.c_int]
_lib.adasap_status_string.restype = ctypes.c_char_p
_lib.adasap_last_error.argtypes = []
_lib.adasap_last_error.restype = ctypes.c_char_p
_lib.adasap_create.argtypes = [_P, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, _P, ctypes.POINTER(_P)]
_lib.adasap_destroy.argtypes = [_P]
_lib.adasap_destroy.restype = None
_lib.adasap_kernel_rows_noalloc.argtypes = [_P, _P, _I64, _P, ctypes.c_int, _P, _P]
_lib.adasap_kernel_rows_noalloc.restype = ctypes.c_int
_lib.adasap_set_precision.argtypes = [_P, ctypes.c_int]
_lib.adasap_set_precision.restype = ctypes.c_int
_lib.adasap_kernel_rows.argtypes = [_P, _P, _I64, _P, ctypes.c_int, _P, _P]
_lib.adasap_solve.argtypes = [_P, _P, ctypes.c_int, ctypes.POINTER(Opts), _P, ctypes.POINTER(Stats), _P]
_lib.adasap_solve_scheduled.argtypes = [_P, _P, ctypes.c_int, ctypes.POINTER(Opts), _P, _P, _P,
                                        ctypes.c_int, _P, _P, ctypes.POINTER(Stats), _P]
_lib.adasap_predict.argtypes = [_P, _P, _I64, _P, ctypes.c_int, _P, _P]
_lib.adasap_hypergrad.argtypes = [_P, _P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), _P]
_lib.adasap_sample.argtypes = [ctypes.c_uint64, _I64, _I64, _I64, ctypes.c_int, _P, _P, _P, _P]
_lib.adasap_solver_begin.argtypes = [_P, _P, ctypes.c_int, ctypes.POINTER(Opts), _P, _P, ctypes.POINTER(_P)]
_lib.adasap_solver_step.argtypes = [_P, ctypes.c_int, _P]
_lib.adasap_solver_residual.argtypes = [_P, ctypes.POINTER(ctypes.c_double), _P]
_lib.adasap_solver_get_w.argtypes = [_P, _P, _P]
_lib.adasap_solver_scalars.argtypes = [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int), _P]
_lib.adasap_solver_graph_kernels.argtypes = [_P, ctypes.POINTER(ctypes.c_int)]
_lib.adasap_solver_graph_kernels.restype = ctypes.c_int
_lib.adasap_solver_diag.argtypes = [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int, _P]
_lib.adasap_solver_diag.restype = ctypes.c_int
_lib.adasap_residual.argtypes = [_P, _P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P]
_lib.adasap_residual.restype = ctypes.c_int
_lib.adasap_solve_batched.argtypes = [ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int,
                                      ctypes.POINTER(Opts), ctypes.POINTER(_P), ctypes.POINTER(Stats), _P]
_lib.adasap_solve_batched.restype = ctypes.c_int
_lib.adasap_rf_prior.argtypes = [_P, _P, _I64, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int, _P, _P]
_lib.adasap_rf_prior.restype = ctypes.c_int
_lib.adasap_pathwise.argtypes = [_P, _P, _P, _I64, _P, _P, _P, _P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(Opts), _P, _P, ctypes.POINTER(Stats), _P]
_lib.adasap_pathwise.restype = ctypes.c_int
_lib.adasap_rmse_nll.argtypes = [_P, _I64, _P, _I64, ctypes.c_int, _P, _I64, ctypes.c_double,
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _P]
_lib.adasap_rmse_nll.restype = ctypes.c_int
_lib.adasap_check_device.argtypes = [_P, ctypes.POINTER(ctypes.c_int), _P]
_lib.adasap_check_device.restype = ctypes.c_int
_lib.adasap_wait_selftest.argtypes = [_P, ctypes.c_uint64, _P]
_lib.adasap_wait_selftest.restype = ctypes.c_int
_lib.adasap_schedule_check.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]
_lib.adasap_schedule_check.restype = ctypes.c_int
_lib.adasap_eval_math.argtypes = [ctypes.c_int, _P, _I64, _P, _P]
_lib.adasap_eval_math.restype = ctypes.c_int
_lib.adasap_solver_get_state.argtypes = [_P, _P, _P, _P, ctypes.POINTER(_I64), _P]
_lib.adasap_solver_get_state.restype = ctypes.c_int
_lib.adasap_solver_set_state.argtypes = [_P, _P, _P, _P, _I64, _P]
_lib.adasap_solver_set_state.restype = ctypes.c_int
_lib.adasap_solver_end.argtypes = [_P]
_lib.adasap_solver_end.restype = None
for _f in ["adasap_solver_begin", "adasap_solver_step", "adasap_solver_residual", "adasap_solver_get_w",
           "adasap_solver_scalars", "adasap_create", "adasap_kernel_rows", "adasap_solve", "adasap_solve_scheduled",
           "adasap_predict", "adasap_hypergrad", "adasap_sample"]:
    getattr(_lib, _f).restype = ctypes.c_int


class AdasapError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        msg = "%s failed: %s (%s)" % (what, STATUS.get(status, status),
                                      _lib.adasap_status_string(status).decode())
        err = _lib.adasap_last_error().decode()
        if err:
            msg += " -- " + err
        super().__init__(msg)


def _check(status, what, allow=()):
    if status != 0 and status not in allow:
        raise AdasapError(status, what)
    return status


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f32(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float32 CUDA tensor" % name)
    return ctypes.c_void_p(t.data_ptr())


def _ptr_any(a, name):
    """Device tensor, or host numpy/tensor (the library copies host buffers)."""
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise TypeError("%s must be contiguous float32" % name)
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("%s must be C-contiguous float32" % name)
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError("%s: unsupported type %r" % (name, type(a)))


def default_opts(n, **kw):
    o = Opts()
    _lib.adasap_default_opts(ctypes.byref(o), int(n))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Context:
    """adasap_create / adasap_destroy around the training inputs X (n x d)."""

    def __init__(self, X, kernel, ell, sigma2, lam, stream=None, precision=None):
        kernel = KERNELS.get(kernel, kernel)
        n, d = X.shape
        h = ctypes.c_void_p()
        _check(_lib.adasap_create(_ptr_any(X, "X"), n, d, int(kernel), float(ell), float(sigma2),
                                  float(lam), _stream(stream), ctypes.byref(h)), "adasap_create")
        self.h = h
        self.n, self.d, self.kernel = n, d, int(kernel)
        self.ell, self.sigma2, self.lam = float(ell), float(sigma2), float(lam)
        if precision is not None:
            self.set_precision(precision)

    def set_precision(self, prec):
        """PREC_FP32 (CUDA-core FP32) or PREC_TF32X3 (tensor-core split distances)."""
        _check(_lib.adasap_set_precision(self.h, int(prec)), "adasap_set_precision")
        self.prec = int(prec)

    def close(self):
        if getattr(self, "h", None):
            _lib.adasap_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def kernel_rows(self, B, W, out=None, stream=None):
        """out (b x s) = K(X_B, X) W."""
        if not (B.is_cuda and B.dtype == torch.int64 and B.is_contiguous()):
            raise TypeError("B must be a contiguous int64 CUDA tensor")
        W2 = W if W.dim() == 2 else W.view(-1, 1)
        b, s = B.numel(), W2.shape[1]
        if out is None:
            out = torch.empty(b, s, device=W.device, dtype=torch.float32)
        _check(_lib.adasap_kernel_rows(self.h, ctypes.c_void_p(B.data_ptr()), b, _dev_f32(W2, "W"), s,
                                       _dev_f32(out, "out"), _stream(stream)), "adasap_kernel_rows")
        return out

    def kernel_rows_noalloc(self, B, W, out, stream=None):
        """adasap_kernel_rows_noalloc: as kernel_rows into a caller-provided `out`,
        allocating nothing (scratch in the library's static device array)."""
        if not (B.is_cuda and B.dtype == torch.int64 and B.is_contiguous()):
            raise TypeError("B must be a contiguous int64 CUDA tensor")
        W2 = W if W.dim() == 2 else W.view(-1, 1)
        _check(_lib.adasap_kernel_rows_noalloc(self.h, ctypes.c_void_p(B.data_ptr()), B.numel(), _dev_f32(W2, "W"),
                                               W2.shape[1], _dev_f32(out, "out"), _stream(stream)),
               "adasap_kernel_rows_noalloc")
        return out

    def solve(self, Y, opts=None, W=None, stream=None, **kw):
        """adasap_solve; Y and W may be host (numpy) or device.  Returns (W, stats, status)."""
        o = opts if opts is not None else default_opts(self.n, **kw)
        s = 1 if Y.ndim == 1 else Y.shape[1]
        if W is None:
            W = torch.zeros(self.n, s, device="cuda", dtype=torch.float32) if isinstance(Y, torch.Tensor) \
                else np.zeros((self.n, s), dtype=np.float32)
        st = Stats()
        status = _lib.adasap_solve(self.h, _ptr_any(Y, "Y"), s, ctypes.byref(o), _ptr_any(W, "W"),
                                   ctypes.byref(st), _stream(stream))
        _check(status, "adasap_solve (stage %d)" % st.status_detail, allow=(7,))
        return W, st.as_dict(), status

    def solve_scheduled(self, Y, B, Omega, v0, opts=None, W=None, trace=True, stream=None, **kw):
        """adasap_solve_scheduled with caller randomness.  Returns (W, trace (T x 2) or None, stats)."""
        T = B.shape[0]
        o = opts if opts is not None else default_opts(self.n, **kw)
        o.b = B.shape[1]
        if Omega is not None:
            o.r = Omega.shape[2]
        s = Y.shape[1]
        if W is None:
            W = torch.zeros(self.n, s, device="cuda", dtype=torch.float32)
        tr = torch.zeros(T, 2, device="cuda", dtype=torch.float64) if trace else None
        st = Stats()
        status = _lib.adasap_solve_scheduled(
            self.h, _ptr_any(Y, "Y"), s, ctypes.byref(o), ctypes.c_void_p(B.data_ptr()),
            ctypes.c_void_p(Omega.data_ptr()) if Omega is not None else None,
            ctypes.c_void_p(v0.data_ptr()), T, _ptr_any(W, "W"),
            ctypes.c_void_p(tr.data_ptr()) if tr is not None else None, ctypes.byref(st),
            _stream(stream))
        _check(status, "adasap_solve_scheduled (stage %d)" % st.status_detail)
        return W, tr, st.as_dict()

    def residual(self, Y, W, stream=None):
        """adasap_residual: ||(K + lambda I) W - Y||_F / ||Y||_F on all rows."""
        Y2 = Y.reshape(Y.shape[0], -1) if Y.ndim == 1 else Y
        W2 = W.reshape(W.shape[0], -1) if W.ndim == 1 else W
        if tuple(Y2.shape) != tuple(W2.shape) or Y2.shape[0] != self.n:
            raise ValueError("Y and W must both be (n, s) with n = %d" % self.n)
        rel = ctypes.c_double()
        _check(_lib.adasap_residual(self.h, _ptr_any(Y2, "Y"), _ptr_any(W2, "W"), Y2.shape[1], ctypes.byref(rel),
                                    _stream(stream)), "adasap_residual")
        return rel.value

    def rf_prior(self, Xq, z, u, phase, theta, stream=None):
        """adasap_rf_prior: random-feature prior draws f(Xq) (m x s); all device tensors."""
        m, q, s = Xq.shape[0], z.shape[0], theta.shape[1]
        F = torch.empty(m, s, device=Xq.device, dtype=torch.float32)
        _check(_lib.adasap_rf_prior(self.h, _dev_f32(Xq, "Xq"), m, _dev_f32(z, "z"),
                                    _dev_f32(u, "u") if u is not None else None, _dev_f32(phase, "phase"),
                                    _dev_f32(theta, "theta"), q, s, _dev_f32(F, "F"), _stream(stream)),
               "adasap_rf_prior")
        return F

    def pathwise(self, y, Xtest, z, u, phase, theta, zeta, with_mean=True, opts=None, W=None, stream=None, **kw):
        """adasap_pathwise: (out (m x (ns + with_mean)), W, stats, status); column 0 = posterior
        mean when with_mean.  All device tensors."""
        m, q, ns = Xtest.shape[0], z.shape[0], theta.shape[1]
        sc = ns + (1 if with_mean else 0)
        o = opts if opts is not None else default_opts(self.n, **kw)
        if W is None:
            W = torch.zeros(self.n, sc, device=y.device, dtype=torch.float32)
        out = torch.empty(m, sc, device=y.device, dtype=torch.float32)
        st = Stats()
        status = _lib.adasap_pathwise(self.h, _dev_f32(y, "y"), _dev_f32(Xtest, "Xtest"), m, _dev_f32(z, "z"),
                                      _dev_f32(u, "u") if u is not None else None, _dev_f32(phase, "phase"),
                                      _dev_f32(theta, "theta"), q, _dev_f32(zeta, "zeta"), ns, int(bool(with_mean)),
                                      ctypes.byref(o), _dev_f32(out, "out"), _dev_f32(W, "W"), ctypes.byref(st),
                                      _stream(stream))
        _check(status, "adasap_pathwise", allow=(7,))
        return out, W, st.as_dict(), status

    def check_device(self, stream=None):
        """adasap_check_device: (status, code) of the bounded device waits since the last check
        (status 6 = ETIMEOUT); clears the record."""
        code = ctypes.c_int()
        status = _lib.adasap_check_device(self.h, ctypes.byref(code), _stream(stream))
        _check(status, "adasap_check_device", allow=(6,))
        return status, code.value

    def wait_selftest(self, limit_ns, stream=None):
        """adasap_wait_selftest: enqueue a bounded wait that nothing completes (test of the failure path)."""
        _check(_lib.adasap_wait_selftest(self.h, int(limit_ns), _stream(stream)), "adasap_wait_selftest")

    def predict(self, Xtest, W, stream=None):
        W2 = W if W.dim() == 2 else W.view(-1, 1)
        m, s = Xtest.shape[0], W2.shape[1]
        out = torch.empty(m, s, device=W.device, dtype=torch.float32)
        _check(_lib.adasap_predict(self.h, _dev_f32(Xtest, "Xtest"), m, _dev_f32(W2, "W"), s,
                                   _dev_f32(out, "out"), _stream(stream)), "adasap_predict")
        return out

    def hypergrad(self, W, G, stream=None):
        W2 = W if W.dim() == 2 else W.view(-1, 1)
        G2 = G if G.dim() == 2 else G.view(-1, 1)
        de, ds = ctypes.c_double(), ctypes.c_double()
        _check(_lib.adasap_hypergrad(self.h, _dev_f32(W2, "W"), _dev_f32(G2, "G"), W2.shape[1],
                                     ctypes.byref(de), ctypes.byref(ds), _stream(stream)), "adasap_hypergrad")
        return de.value, ds.value


class Solver:
    """adasap_solver_begin/step/residual/get_w/scalars/end around one Context."""

    def __init__(self, context, Y, opts=None, W0=None, stream=None, **kw):
        self.context = context
        self.o = opts if opts is not None else default_opts(context.n, **kw)
        self.s = 1 if Y.ndim == 1 else Y.shape[1]
        h = ctypes.c_void_p()
        _check(_lib.adasap_solver_begin(context.h, _ptr_any(Y, "Y"), self.s, ctypes.byref(self.o),
                                        _ptr_any(W0, "W0") if W0 is not None else None, _stream(stream),
                                        ctypes.byref(h)), "adasap_solver_begin")
        self.h = h

    def step(self, iters=1, stream=None):
        _check(_lib.adasap_solver_step(self.h, int(iters), _stream(stream)), "adasap_solver_step")

    def residual(self, stream=None):
        rel = ctypes.c_double()
        _check(_lib.adasap_solver_residual(self.h, ctypes.byref(rel), _stream(stream)), "adasap_solver_residual")
        return rel.value

    def get_w(self, out=None, stream=None):
        if out is None:
            out = torch.empty(self.context.n, self.s, device="cuda", dtype=torch.float32)
        _check(_lib.adasap_solver_get_w(self.h, _ptr_any(out, "W"), _stream(stream)), "adasap_solver_get_w")
        return out

    def get_state(self, stream=None):
        """adasap_solver_get_state: (W, V, Z, t) as device tensors and an int."""
        mk = lambda: torch.empty(self.context.n, self.s, device="cuda", dtype=torch.float32)
        W, V, Z = mk(), mk(), mk()
        t = _I64()
        _check(_lib.adasap_solver_get_state(self.h, _ptr_any(W, "W"), _ptr_any(V, "V"), _ptr_any(Z, "Z"),
                                            ctypes.byref(t), _stream(stream)), "adasap_solver_get_state")
        return W, V, Z, t.value

    def set_state(self, W, V, Z, t, stream=None):
        """adasap_solver_set_state: resume from (W, V, Z, t) (host or device arrays)."""
        _check(_lib.adasap_solver_set_state(self.h, _ptr_any(W, "W"), _ptr_any(V, "V"), _ptr_any(Z, "Z"), int(t),
                                            _stream(stream)), "adasap_solver_set_state")

    def scalars(self, stream=None):
        eta, rho, st = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        _check(_lib.adasap_solver_scalars(self.h, ctypes.byref(eta), ctypes.byref(rho), ctypes.byref(st),
                                          _stream(stream)), "adasap_solver_scalars")
        return eta.value, rho.value, st.value

    DIAG = ["delta", "rho", "eta", "lam_hat", "chol_retries", "jacobi_sweeps", "status", "detail", "t", "tc_err"]

    def diag(self, stream=None):
        out = (ctypes.c_double * len(self.DIAG))()
        _check(_lib.adasap_solver_diag(self.h, out, len(self.DIAG), _stream(stream)), "adasap_solver_diag")
        return dict(zip(self.DIAG, list(out)))

    def graph_kernels(self):
        k = ctypes.c_int()
        _check(_lib.adasap_solver_graph_kernels(self.h, ctypes.byref(k)), "adasap_solver_graph_kernels")
        return k.value

    def close(self):
        if getattr(self, "h", None):
            _lib.adasap_solver_end(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(contexts, Ys, opts=None, Ws=None, stream=None):
    """adasap_solve_batched over independent systems (contexts[i], Ys[i]); Ys / Ws host or
    device (n_i x s).  opts: list of Opts (default: default_opts(n_i)).  Returns
    (Ws, list of stats dicts, status)."""
    k = len(contexts)
    if len(Ys) != k or k == 0:
        raise ValueError("one Y per context")
    Y2 = [Y.reshape(Y.shape[0], -1) if Y.ndim == 1 else Y for Y in Ys]
    s = Y2[0].shape[1]
    for ctx, Y in zip(contexts, Y2):
        if Y.shape[0] != ctx.n or Y.shape[1] != s:
            raise ValueError("Y_i must be (n_i, s) with one s for all systems")
    if opts is None:
        opts = [default_opts(ctx.n) for ctx in contexts]
    if Ws is None:
        Ws = [torch.zeros(ctx.n, s, device="cuda", dtype=torch.float32) if isinstance(Y, torch.Tensor)
              else np.zeros((ctx.n, s), dtype=np.float32) for ctx, Y in zip(contexts, Y2)]
    ctx_arr = (ctypes.c_void_p * k)(*[ctx.h.value for ctx in contexts])
    y_arr = (ctypes.c_void_p * k)(*[_ptr_any(Y, "Y").value for Y in Y2])
    w_arr = (ctypes.c_void_p * k)(*[_ptr_any(W, "W").value for W in Ws])
    o_arr = (Opts * k)(*opts)
    st_arr = (Stats * k)()
    status = _lib.adasap_solve_batched(k, ctx_arr, y_arr, s, o_arr, w_arr, st_arr, _stream(stream))
    _check(status, "adasap_solve_batched", allow=(7,))
    return Ws, [st.as_dict() for st in st_arr], status


def rmse_nll(mean, samples, ytest, noise, stream=None):
    """adasap_rmse_nll on device tensors: mean (m,) or a column view, samples (m, s) (row stride
    may exceed s), ytest (m,).  Returns (rmse, nll)."""
    m, s = samples.shape
    for t, name in ((mean, "mean"), (samples, "samples"), (ytest, "ytest")):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32):
            raise TypeError("%s must be a float32 CUDA tensor" % name)
    if samples.stride(1) != 1 or ytest.stride(0) != 1:
        raise TypeError("samples rows and ytest must be contiguous")
    ldm = mean.stride(0)
    rm, nl = ctypes.c_double(), ctypes.c_double()
    _check(_lib.adasap_rmse_nll(ctypes.c_void_p(mean.data_ptr()), ldm, ctypes.c_void_p(samples.data_ptr()),
                                samples.stride(0), s, ctypes.c_void_p(ytest.data_ptr()), m, float(noise),
                                ctypes.byref(rm), ctypes.byref(nl), _stream(stream)), "adasap_rmse_nll")
    return rm.value, nl.value


def schedule_check(m, ncols, max_ctas=0):
    """adasap_schedule_check (host only): (status, nsplit, flat) of the single-RHS tensor-core
    product's work schedule; status is ADASAP_OK (0) when every tile and (row, slot) is covered once."""
    ns, fl = ctypes.c_int(), ctypes.c_int()
    st = _lib.adasap_schedule_check(int(m), int(ncols), int(max_ctas), ctypes.byref(ns), ctypes.byref(fl))
    return st, ns.value, bool(fl.value)


def eval_math(fn, x, stream=None):
    """adasap_eval_math: f(x) element by element on the device (fn 0: the FMA-pipe square
    root of the Matern epilogues, 1: sqrt.approx)."""
    xt = x.contiguous()
    out = torch.empty_like(xt)
    _check(_lib.adasap_eval_math(int(fn), _dev_f32(xt, "x"), xt.numel(), ctypes.c_void_p(out.data_ptr()),
                                 _stream(stream)), "adasap_eval_math")
    return out


def measure_pipes(stream=None):
    """adasap_measure_pipes: measured ex2, rsqrt, FP32-FMA and sqrt issue rates (per SM per cycle)."""
    out = (ctypes.c_double * 4)()
    _check(_lib.adasap_measure_pipes(out, 4, _stream(stream)), "adasap_measure_pipes")
    return {"ex2": out[0], "rsqrt": out[1], "ffma": out[2], "sqrt": out[3]}


def sample(seed, t, n, b, r, stream=None):
    """adasap_sample: (B int64 (b,), Omega (b, r), v0 (b,)) on the current CUDA device."""
    B = torch.empty(b, device="cuda", dtype=torch.int64)
    Om = torch.empty(b, max(r, 1), device="cuda", dtype=torch.float32)
    v0 = torch.empty(b, device="cuda", dtype=torch.float32)
    _check(_lib.adasap_sample(int(seed), int(t), int(n), int(b), int(r), ctypes.c_void_p(B.data_ptr()),
                              ctypes.c_void_p(Om.data_ptr()) if r > 0 else None,
                              ctypes.c_void_p(v0.data_ptr()), _stream(stream)), "adasap_sample")
    return B, Om[:, :r], v0


class KernelMatmul(torch.autograd.Function):
    """y = K(X, X; ell, sigma2) W with the hand-written adjoint kernel for (ell, sigma2).

    Forward and the W-gradient are adasap_kernel_rows over all rows (K is
    symmetric, so dL/dW = K G); the (ell, sigma2) gradients are adasap_hypergrad.
    ``ell`` and ``sigma2`` must equal the context's values (the context's
    device copy of X is scaled by ell).
    """

    @staticmethod
    def forward(ctx, context, W, ell, sigma2):
        if abs(float(ell) - context.ell) > 1e-6 * context.ell or abs(float(sigma2) - context.sigma2) > 1e-6 * context.sigma2:
            raise ValueError("ell / sigma2 differ from the context's; build a new Context")
        rows = torch.arange(context.n, device=W.device, dtype=torch.int64)
        ctx.context = context
        ctx.save_for_backward(W, rows)
        return context.kernel_rows(rows, W.contiguous())

    @staticmethod
    def backward(ctx, G):
        W, rows = ctx.saved_tensors
        context = ctx.context
        G = G.contiguous()
        gW = context.kernel_rows(rows, G) if ctx.needs_input_grad[1] else None
        d_ell = d_s2 = None
        if ctx.needs_input_grad[2] or ctx.needs_input_grad[3]:
            de, ds = context.hypergrad(W.contiguous(), G)
            d_ell = torch.tensor(de, dtype=torch.float32, device=W.device)
            d_s2 = torch.tensor(ds, dtype=torch.float32, device=W.device)
        return None, gW, d_ell, d_s2
