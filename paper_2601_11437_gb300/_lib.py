"""ctypes declarations of libfbt.so (include/fbt.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfbt.so")

c_double_p = C.POINTER(C.c_double)


class FbtOpts(C.Structure):
    _fields_ = [("jitter", C.c_double), ("nb", C.c_int), ("reorder", C.c_int),
                ("with_derivatives", C.c_int), ("device", C.c_int), ("precision", C.c_int),
                ("mixed_tol", C.c_double)]


class FbtBtOpts(C.Structure):
    _fields_ = [("armijo_c", C.c_double), ("rho", C.c_double), ("slack", C.c_double),
                ("grad_tol", C.c_double), ("nm_ftol", C.c_double), ("max_ll_calls", C.c_int),
                ("max_grad_calls", C.c_int), ("nm_max_calls", C.c_int), ("max_halvings", C.c_int),
                ("polish_step", C.c_double)]


class FbtState(C.Structure):
    _fields_ = [("theta", C.c_double * 3), ("phi", C.c_double * 3), ("loglik", C.c_double),
                ("score", C.c_double * 3), ("fisher", C.c_double * 9), ("n_ll", C.c_int),
                ("n_grad", C.c_int), ("iter", C.c_int), ("state", C.c_int), ("halvings", C.c_int),
                ("polish_iter", C.c_int), ("theta_mixed", C.c_double * 3)]


class FbtKernelStat(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_longlong), ("ms", C.c_double),
                ("flops", C.c_double), ("bytes", C.c_double)]


# name -> (restype, argtypes)
SIGNATURES = {
    "fbt_default_opts": (None, [C.POINTER(FbtOpts)]),
    "fbt_workspace_bytes": (C.c_size_t, [C.c_longlong, C.POINTER(FbtOpts)]),
    "fbt_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                             C.c_longlong, C.POINTER(FbtOpts), C.c_void_p, C.c_size_t, C.c_void_p]),
    "fbt_set_field": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "mle_loglik": (C.c_int, [C.c_void_p, c_double_p, c_double_p]),
    "mle_eval": (C.c_int, [C.c_void_p, c_double_p, c_double_p, c_double_p, c_double_p]),
    "mle_loglik_grad": (C.c_int, [C.c_void_p, c_double_p, c_double_p, c_double_p]),
    "fbt_default_bt_opts": (None, [C.POINTER(FbtBtOpts)]),
    "fisher_bt_start": (C.c_int, [C.c_void_p, c_double_p, c_double_p, c_double_p,
                                  C.POINTER(FbtBtOpts), C.POINTER(FbtState)]),
    "fisher_bt_step": (C.c_int, [C.c_void_p, C.POINTER(FbtState), C.POINTER(FbtBtOpts)]),
    "fisher_bt_run": (C.c_int, [C.c_void_p, c_double_p, c_double_p, c_double_p,
                                C.POINTER(FbtBtOpts), C.POINTER(FbtState)]),
    "mle_eval_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, c_double_p, C.c_int, C.c_int, c_double_p,
                                 C.POINTER(C.c_int), C.c_int]),
    "fisher_bt_start_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, c_double_p, c_double_p, c_double_p,
                                        C.POINTER(FbtBtOpts), C.POINTER(FbtState), C.POINTER(C.c_int), C.c_int]),
    "fisher_bt_step_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(FbtState),
                                       C.POINTER(FbtBtOpts), C.POINTER(C.c_int), C.c_int]),
    "fisher_bt_run_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, c_double_p, c_double_p, c_double_p,
                                      C.POINTER(FbtBtOpts), C.POINTER(FbtState), C.POINTER(C.c_int), C.c_int]),
    "fbt_tune_batch_threads": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, c_double_p, C.POINTER(C.c_int), C.c_int,
                                         C.POINTER(C.c_int), c_double_p]),
    "fbt_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, c_double_p, C.c_int, C.POINTER(FbtOpts),
                               c_double_p, C.POINTER(C.c_int)]),
    "fbt_set_graphs": (C.c_int, [C.c_void_p, C.c_int]),
    "fbt_graph_count": (C.c_int, [C.c_void_p]),
    "fbt_set_mixed_tol": (C.c_int, [C.c_void_p, C.c_double]),
    "fbt_get_mixed_tol": (C.c_double, [C.c_void_p]),
    "fbt_mixed_counts": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.c_int]),
    "fbt_set_spin_budget": (C.c_int, [C.c_void_p, C.c_longlong]),
    "fbt_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "fbt_profile_read": (C.c_int, [C.c_void_p, C.POINTER(FbtKernelStat), C.c_int, C.POINTER(C.c_int)]),
    "fbt_launch_count": (C.c_longlong, [C.c_void_p, C.c_int]),
    "fbt_factor_reuses": (C.c_longlong, [C.c_void_p]),
    "fbt_transfer_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.c_int]),
    "fbt_geometry": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                               C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "fbt_copy_slab": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "fbt_copy_perm": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong)]),
    "fbt_generate": (C.c_int, [C.c_void_p, c_double_p, C.c_int]),
    "fbt_noalloc_max_n": (C.c_longlong, []),
    "fbt_loglik_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_longlong, c_double_p, C.c_double,
                                     c_double_p, C.c_void_p]),
    "fbt_destroy": (None, [C.c_void_p]),
    "fbt_strerror": (C.c_char_p, [C.c_int]),
    "fbt_last_cuda_error": (C.c_char_p, []),
}

_LIB = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libfbt.so (built by paper_2601_11437_gb300.build); raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2601_11437_gb300.build` "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib
