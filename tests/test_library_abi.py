"""CPU-side checks of the C ABI: libfbt.so builds for sm_103a, loads, and exports every entry
point include/fbt.h declares (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fbt.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text)
    keywords = {"if", "while", "for", "sizeof", "return", "defined"}
    types = {"size_t"}
    return sorted({n for n in names if n not in keywords and n not in types})


@pytest.fixture(scope="module")
def lib():
    from paper_2601_11437_gb300 import build, _lib
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fbt_create", "mle_loglik", "mle_eval", "fisher_bt_step", "fisher_bt_run",
                     "fbt_destroy", "fbt_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_same_names(lib):
    from paper_2601_11437_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(declared_functions())


def test_host_only_entry_points(lib):
    from paper_2601_11437_gb300 import _lib
    L = _lib.load()
    opts = _lib.FbtOpts()
    L.fbt_default_opts(ctypes.byref(opts))
    assert (opts.jitter, opts.nb, opts.reorder, opts.with_derivatives) == (1e-8, 128, 1, 1)
    bt = _lib.FbtBtOpts()
    L.fbt_default_bt_opts(ctypes.byref(bt))
    assert (bt.armijo_c, bt.rho, bt.slack, bt.grad_tol, bt.nm_ftol) == (0.001, 0.5, 0.001, 0.001, 1e-9)
    assert (bt.max_ll_calls, bt.max_grad_calls) == (60, 20)
    # workspace size: 3 slabs of T(T+1)/2 tiles of nb^2 doubles dominate
    n, nb = 1000, 128
    T = (n + nb - 1) // nb
    ws = L.fbt_workspace_bytes(n, ctypes.byref(opts))
    assert ws >= 3 * T * (T + 1) // 2 * nb * nb * 8
    opts.nb = 96
    assert L.fbt_workspace_bytes(n, ctypes.byref(opts)) == 0
    assert L.fbt_workspace_bytes(0, None) == 0
    assert L.fbt_strerror(2).decode().startswith("covariance matrix not positive definite")
    # argument checks happen before any device call
    h = ctypes.c_void_p()
    assert L.fbt_create(ctypes.byref(h), None, 0, None, 0, 10, None, None, 0, None) == 7
    assert L.mle_loglik(None, None, None) == 7
    assert L.fisher_bt_step(None, None, None) == 7


def test_noalloc_entry_point_signature_and_argument_checks(lib):
    """The allocation-free entry point's exports, signatures in the binding, and the argument
    rejections that happen before any CUDA call (so they run without a GPU)."""
    from paper_2601_11437_gb300 import _lib
    L = _lib.load()
    assert "fbt_noalloc_max_n" in declared_functions() and "fbt_loglik_noalloc" in declared_functions()
    res, args = _lib.SIGNATURES["fbt_noalloc_max_n"]
    assert res is ctypes.c_longlong and args == []
    res, args = _lib.SIGNATURES["fbt_loglik_noalloc"]
    assert res is ctypes.c_int
    assert args == [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong,
                    ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                    ctypes.c_void_p]
    max_n = L.fbt_noalloc_max_n()
    assert max_n == 1024
    import numpy as np
    locs = np.zeros((max_n + 1, 2))
    z = np.zeros(max_n + 1)
    th = (ctypes.c_double * 3)(1.0, 0.1, 0.5)
    out = ctypes.c_double(0.0)
    pl, pz = locs.ctypes.data_as(ctypes.c_void_p), z.ctypes.data_as(ctypes.c_void_p)
    ARG, DOMAIN = 7, 1
    assert L.fbt_loglik_noalloc(pl, pz, 0, 0, th, 1e-8, ctypes.byref(out), None) == ARG          # n < 1
    assert L.fbt_loglik_noalloc(pl, pz, 0, max_n + 1, th, 1e-8, ctypes.byref(out), None) == ARG  # n > max
    assert L.fbt_loglik_noalloc(None, pz, 0, 10, th, 1e-8, ctypes.byref(out), None) == ARG        # NULL
    assert L.fbt_loglik_noalloc(pl, None, 0, 10, th, 1e-8, ctypes.byref(out), None) == ARG
    assert L.fbt_loglik_noalloc(pl, pz, 0, 10, None, 1e-8, ctypes.byref(out), None) == ARG
    assert L.fbt_loglik_noalloc(pl, pz, 0, 10, th, 1e-8, None, None) == ARG
    assert L.fbt_loglik_noalloc(pl, pz, 0, 10, th, -1e-8, ctypes.byref(out), None) == ARG         # jitter < 0
    assert L.fbt_loglik_noalloc(pl, pz, 0, 10, th, float("nan"), ctypes.byref(out), None) == ARG
    assert L.fbt_loglik_noalloc(pl, pz, 0, 10, th, float("inf"), ctypes.byref(out), None) == ARG
    bad = (ctypes.c_double * 3)(1.0, 0.0, 0.5)
    assert L.fbt_loglik_noalloc(pl, pz, 0, 10, bad, 1e-8, ctypes.byref(out), None) == DOMAIN
    assert out.value == float("-inf")
