"""CPU checks of the C-ABI boundary: the library loads, exports every declared
symbol, and its host-only entry points behave (no GPU work is issued)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "adasap.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(adasap_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def cdll():
    from paper_2505_13723_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    fns = declared_functions()
    for name in ["adasap_create", "adasap_kernel_rows", "adasap_solve", "adasap_predict",
                 "adasap_hypergrad", "adasap_destroy"]:
        assert name in fns


def test_library_exports_every_declared_symbol(cdll):
    missing = [f for f in declared_functions() if not hasattr(cdll, f)]
    assert not missing, missing


def test_binding_lists_exactly_the_declared_symbols(cdll):
    from paper_2505_13723_b300 import binding
    assert sorted(binding.SYMBOLS) == declared_functions()


def test_default_opts_layout_and_paper_defaults(cdll):
    from paper_2505_13723_b300 import binding
    o = binding.default_opts(1 << 20)
    assert o.b == (1 << 20) // 100          # b = n/100 (App. D.2)
    assert o.r == 100                       # r = 100 (App. D.2)
    assert o.power_iters == 10              # 10 powering iterations (App. C.3)
    assert o.mu == 0 and o.nu == 0          # => mu = lambda, nu = n/b (Sec. 4.2)
    assert o.precond == 0 and o.literal == 0
    small = binding.default_opts(50)
    assert small.b == 50 and small.r == 50


def test_invalid_arguments_are_rejected_on_the_host(cdll):
    from paper_2505_13723_b300 import binding
    lib = binding._lib
    h = ctypes.c_void_p()
    x = (ctypes.c_float * 10)()
    # d > 64, non-positive hyperparameters, bad kernel id: EINVAL before any GPU call
    assert lib.adasap_create(ctypes.cast(x, ctypes.c_void_p), 1, 65, 0, 1.0, 1.0, 1.0, None, ctypes.byref(h)) == 1
    assert lib.adasap_create(ctypes.cast(x, ctypes.c_void_p), 10, 1, 0, -1.0, 1.0, 1.0, None, ctypes.byref(h)) == 1
    assert lib.adasap_create(ctypes.cast(x, ctypes.c_void_p), 10, 1, 7, 1.0, 1.0, 1.0, None, ctypes.byref(h)) == 1
    assert lib.adasap_kernel_rows(None, None, 1, None, 1, None, None) == 1
    assert lib.adasap_solve(None, None, 1, None, None, None, None) == 1
    assert lib.adasap_sample(0, 0, 10, 11, 1, None, None, None, None) == 1   # b > n
    assert lib.adasap_status_string(4) == b"Cholesky of an r x r core failed"
