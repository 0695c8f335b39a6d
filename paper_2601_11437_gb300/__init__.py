"""GB300-native Fisher-BT: exact Matern log-likelihood, score and Fisher information on the GPU.

Python binding of libfbt.so (include/fbt.h) with the same entry-point names.  It only marshals
arguments: every step of an evaluation runs in the library's CUDA kernels, and importing or
calling the binding without the built library (or without a GPU) raises; there is no CPU
fallback.  PyTorch provides the device workspace (caching allocator) and the CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import _lib
from ._lib import FbtBtOpts, FbtOpts, FbtState, FbtKernelStat  # noqa: F401

FBT_OK, FBT_ERR_DOMAIN, FBT_ERR_NOT_PD, FBT_ERR_BESSEL = 0, 1, 2, 3
FBT_ERR_TIMEOUT, FBT_ERR_CUDA, FBT_ERR_OOM, FBT_ERR_ARG, FBT_ERR_STATE = 4, 5, 6, 7, 8
RUNNING, CONVERGED, SHIFT, DONE_NM, FAILED = 0, 1, 2, 3, -1
_SOFT = (FBT_ERR_DOMAIN, FBT_ERR_NOT_PD, FBT_ERR_BESSEL)


class FbtError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        lib = _lib.load()
        msg = lib.fbt_strerror(status).decode()
        if status == FBT_ERR_CUDA:
            msg += ": " + lib.fbt_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


def _check(status: int, where: str) -> int:
    if status != FBT_OK and status not in _SOFT:
        raise FbtError(status, where)
    return status


def _dbl3(v) -> C.Array:
    a = (C.c_double * 3)(*[float(t) for t in v])
    return a


class Context:
    """A libfbt context: device copies of locations and field plus the tile workspace."""

    def __init__(self, handle, n, workspace, opts):
        self.handle = C.c_void_p(handle)
        self.n = n
        self.workspace = workspace          # torch tensor keeping the device memory alive
        self.opts = opts

    def geometry(self):
        n, npad, nb, T = C.c_longlong(), C.c_longlong(), C.c_int(), C.c_int()
        _check(_lib.load().fbt_geometry(self.handle, C.byref(n), C.byref(npad), C.byref(nb), C.byref(T)), "fbt_geometry")
        return dict(n=n.value, npad=npad.value, nb=nb.value, tiles=T.value)

    def __del__(self):
        try:
            fbt_destroy(self)
        except Exception:
            pass


PREC_FP64, PREC_FP64_EMULATED, PREC_MIXED = 0, 1, 2


def fbt_create(locs, z, *, nb: int = 128, jitter: float = 1e-8, reorder: bool = True,
               with_derivatives: bool = True, device: int = 0, stream=None,
               workspace: str = "torch", precision: int = PREC_FP64, mixed_tol: float = 1e-12) -> Context:
    """fbt_create: locs (n, 2) and z (n,) as float64 numpy arrays (host) or CUDA tensors (device)."""
    import torch
    lib = _lib.load()
    if not torch.cuda.is_available():
        raise FbtError(FBT_ERR_CUDA, "fbt_create (no CUDA device)")
    opts = FbtOpts()
    lib.fbt_default_opts(C.byref(opts))
    opts.nb, opts.jitter, opts.reorder = nb, jitter, int(bool(reorder))
    opts.with_derivatives, opts.device = int(bool(with_derivatives)), device
    opts.precision = int(precision)
    opts.mixed_tol = float(mixed_tol)

    def ptr(a, shape):
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or a.device.type != "cuda" or not a.is_contiguous():
                raise ValueError("device inputs must be contiguous float64 CUDA tensors")
            if tuple(a.shape) != shape:
                raise ValueError(f"expected shape {shape}, got {tuple(a.shape)}")
            return C.c_void_p(a.data_ptr()), 1, a
        arr = np.ascontiguousarray(a, dtype=np.float64)
        if arr.shape != shape:
            raise ValueError(f"expected shape {shape}, got {arr.shape}")
        return arr.ctypes.data_as(C.c_void_p), 0, arr

    n = int(z.shape[0])
    pl, ld, keep_l = ptr(locs, (n, 2))
    pz, zd, keep_z = ptr(z, (n,))
    nbytes = lib.fbt_workspace_bytes(n, C.byref(opts))
    if nbytes == 0:
        raise FbtError(FBT_ERR_ARG, "fbt_workspace_bytes")
    ws, wsp = None, None
    if workspace == "torch":
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=f"cuda:{device}")
        base = ws.data_ptr()
        wsp = C.c_void_p((base + 255) & ~255)
    if stream is None:
        stream = torch.cuda.current_stream(device).cuda_stream
    h = C.c_void_p()
    st = lib.fbt_create(C.byref(h), pl, ld, pz, zd, n, C.byref(opts), wsp, nbytes if ws is not None else 0,
                        C.c_void_p(stream))
    if st != FBT_OK:
        raise FbtError(st, "fbt_create")
    del keep_l, keep_z
    return Context(h.value, n, ws, opts)


def fbt_set_field(ctx: Context, z) -> None:
    import torch
    if isinstance(z, torch.Tensor):
        _check(_lib.load().fbt_set_field(ctx.handle, C.c_void_p(z.data_ptr()), 1), "fbt_set_field")
    else:
        arr = np.ascontiguousarray(z, dtype=np.float64)
        _check(_lib.load().fbt_set_field(ctx.handle, arr.ctypes.data_as(C.c_void_p), 0), "fbt_set_field")


def mle_loglik(ctx: Context, theta) -> float:
    """Algorithm 2: l(theta); -inf for theta outside the domain or a non-PD covariance."""
    out = C.c_double()
    _check(_lib.load().mle_loglik(ctx.handle, _dbl3(theta), C.byref(out)), "mle_loglik")
    return out.value


def mle_eval(ctx: Context, theta):
    """Algorithm 3: (l, score (3,), Fisher (3, 3)); raises on a soft failure."""
    ll, g, I = C.c_double(), (C.c_double * 3)(), (C.c_double * 9)()
    st = _lib.load().mle_eval(ctx.handle, _dbl3(theta), C.byref(ll), g, I)
    if st != FBT_OK:
        raise FbtError(st, "mle_eval")
    return ll.value, np.array(g[:]), np.array(I[:]).reshape(3, 3)


def mle_loglik_grad(ctx: Context, theta):
    """Adjoint: (l, grad l (3,)) through Sigma^-1 with the partials regenerated on the fly."""
    ll, g = C.c_double(), (C.c_double * 3)()
    st = _lib.load().mle_loglik_grad(ctx.handle, _dbl3(theta), C.byref(ll), g)
    if st != FBT_OK:
        raise FbtError(st, "mle_loglik_grad")
    return ll.value, np.array(g[:])


class MaternLogLik:
    """torch.autograd.Function for l(theta): forward runs Algorithm 2 (mle_loglik), backward the
    adjoint (mle_loglik_grad), which reuses the forward's Cholesky factor.  Use
    MaternLogLik.apply(ctx, theta_tensor) with a float64 tensor of shape (3,)."""

    _fn = None

    @classmethod
    def apply(cls, ctx: Context, theta):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(fctx, theta_t, handle_holder):
                    th = [float(v) for v in theta_t.detach().cpu().tolist()]
                    fctx.th = th
                    fctx.holder = handle_holder
                    return torch.tensor(mle_loglik(handle_holder, th), dtype=torch.float64)

                @staticmethod
                def backward(fctx, grad_out):
                    _, g = mle_loglik_grad(fctx.holder, fctx.th)
                    return grad_out * torch.tensor(g, dtype=torch.float64), None

            cls._fn = _F
        return cls._fn.apply(theta, ctx)


def default_bt_opts() -> FbtBtOpts:
    bt = FbtBtOpts()
    _lib.load().fbt_default_bt_opts(C.byref(bt))
    return bt


def _opt3(v):
    return None if v is None else _dbl3(v)


def fisher_bt_start(ctx: Context, theta0=None, theta_lo=None, theta_hi=None, bt=None) -> FbtState:
    st = FbtState()
    bt = bt or default_bt_opts()
    s = _lib.load().fisher_bt_start(ctx.handle, _opt3(theta0), _opt3(theta_lo), _opt3(theta_hi), C.byref(bt), C.byref(st))
    _check(s, "fisher_bt_start")
    return st


def fisher_bt_step(ctx: Context, state: FbtState, bt=None) -> FbtState:
    bt = bt or default_bt_opts()
    s = _lib.load().fisher_bt_step(ctx.handle, C.byref(state), C.byref(bt))
    _check(s, "fisher_bt_step")
    return state


def fisher_bt_run(ctx: Context, theta0=None, theta_lo=None, theta_hi=None, bt=None) -> FbtState:
    st = FbtState()
    bt = bt or default_bt_opts()
    s = _lib.load().fisher_bt_run(ctx.handle, _opt3(theta0), _opt3(theta_lo), _opt3(theta_hi), C.byref(bt), C.byref(st))
    _check(s, "fisher_bt_run")
    return st


FBT_BATCH_LOGLIK, FBT_BATCH_EVAL = 0, 1


def _handles(ctxs):
    return (C.c_void_p * len(ctxs))(*[c.handle.value for c in ctxs])


def _rows3(v, rows):
    """(pointer, owner) of a contiguous (rows, 3) float64 copy of v, or (None, None)."""
    if v is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(rows, 3))
    return a.ctypes.data_as(_lib.c_double_p), a


def mle_eval_batch(ctxs, thetas, *, full: bool = True, nthreads: int = 0):
    """k candidates for each of F fields (thetas: (F, k, 3)).  full: returns (l (F, k),
    score (F, k, 3), fisher (F, k, 3, 3), status (F, k)); else (l (F, k), status (F, k))."""
    F = len(ctxs)
    th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).reshape(F, -1, 3))
    k = th.shape[1]
    stride = 13 if full else 1
    out = np.zeros((F, k, stride))
    status = np.zeros((F, k), dtype=np.int32)
    s = _lib.load().mle_eval_batch(_handles(ctxs), F, th.ctypes.data_as(_lib.c_double_p), k,
                                   FBT_BATCH_EVAL if full else FBT_BATCH_LOGLIK,
                                   out.ctypes.data_as(_lib.c_double_p),
                                   status.ctypes.data_as(C.POINTER(C.c_int)), nthreads)
    if s != FBT_OK:
        raise FbtError(s, "mle_eval_batch")
    if full:
        return out[..., 0], out[..., 1:4], out[..., 4:13].reshape(F, k, 3, 3), status
    return out[..., 0], status


def _batch_states(F):
    return (FbtState * F)(), np.zeros(F, dtype=np.int32)


def fisher_bt_start_batch(ctxs, theta0s=None, theta_lo=None, theta_hi=None, bt=None, nthreads: int = 0):
    """fisher_bt_start per field; returns (states (FbtState array), status (F,))."""
    F = len(ctxs)
    states, status = _batch_states(F)
    (p0, a0), (pl, al), (ph, ah) = _rows3(theta0s, F), _rows3(theta_lo, F), _rows3(theta_hi, F)
    bt = bt or default_bt_opts()
    s = _lib.load().fisher_bt_start_batch(_handles(ctxs), F, p0, pl, ph, C.byref(bt), states,
                                          status.ctypes.data_as(C.POINTER(C.c_int)), nthreads)
    if s != FBT_OK:
        raise FbtError(s, "fisher_bt_start_batch")
    return states, status


def fisher_bt_step_batch(ctxs, states, bt=None, nthreads: int = 0):
    """One Fisher-BT step of every field still running (in place); returns status (F,)."""
    F = len(ctxs)
    status = np.zeros(F, dtype=np.int32)
    bt = bt or default_bt_opts()
    s = _lib.load().fisher_bt_step_batch(_handles(ctxs), F, states, C.byref(bt),
                                         status.ctypes.data_as(C.POINTER(C.c_int)), nthreads)
    if s != FBT_OK:
        raise FbtError(s, "fisher_bt_step_batch")
    return status


def fisher_bt_run_batch(ctxs, theta0s=None, theta_lo=None, theta_hi=None, bt=None, nthreads: int = 0):
    """Algorithm 1 end to end for every field; returns (states, status (F,))."""
    F = len(ctxs)
    states, status = _batch_states(F)
    (p0, a0), (pl, al), (ph, ah) = _rows3(theta0s, F), _rows3(theta_lo, F), _rows3(theta_hi, F)
    bt = bt or default_bt_opts()
    s = _lib.load().fisher_bt_run_batch(_handles(ctxs), F, p0, pl, ph, C.byref(bt), states,
                                        status.ctypes.data_as(C.POINTER(C.c_int)), nthreads)
    if s != FBT_OK:
        raise FbtError(s, "fisher_bt_run_batch")
    return states, status


def fbt_tune_batch_threads(ctxs, thetas, candidates=(8, 16, 32, 64)):
    """Autotuner: the fastest host-thread count of the batched entry points on these fields;
    returns (best, {candidate: seconds})."""
    F = len(ctxs)
    th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).reshape(F, 3))
    cand = (C.c_int * len(candidates))(*candidates)
    secs = (C.c_double * len(candidates))()
    best = C.c_int()
    _check(_lib.load().fbt_tune_batch_threads(_handles(ctxs), F, th.ctypes.data_as(_lib.c_double_p), cand,
                                              len(candidates), C.byref(best), secs), "fbt_tune_batch_threads")
    return best.value, {c: secs[i] for i, c in enumerate(candidates)}


def fbt_autotune(locs, z, theta, *, precision: int = PREC_FP64_EMULATED, reps: int = 2, device: int = 0):
    """Autotuner: the faster FP64-accurate configuration (precision, nb) for a field of this size;
    returns (precision, nb, {"fp64_nb64": s, "emulated_nb128": s}, cached)."""
    lib = _lib.load()
    opts = FbtOpts()
    lib.fbt_default_opts(C.byref(opts))
    opts.precision, opts.device = int(precision), device
    locs = np.ascontiguousarray(locs, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    secs = (C.c_double * 2)()
    cached = C.c_int()
    _check(lib.fbt_autotune(locs.ctypes.data_as(C.c_void_p), z.ctypes.data_as(C.c_void_p), len(z), _dbl3(theta),
                            int(reps), C.byref(opts), secs, C.byref(cached)), "fbt_autotune")
    return opts.precision, opts.nb, {"fp64_nb64": secs[0], "emulated_nb128": secs[1]}, bool(cached.value)


def fbt_destroy(ctx: Context) -> None:
    if ctx.handle and ctx.handle.value:
        _lib.load().fbt_destroy(ctx.handle)
        ctx.handle = C.c_void_p(None)
        ctx.workspace = None


def fbt_set_graphs(ctx: Context, enable: bool) -> None:
    """Replay evaluations as captured CUDA graphs (default) or launch every kernel directly."""
    _check(_lib.load().fbt_set_graphs(ctx.handle, 1 if enable else 0), "fbt_set_graphs")


def fbt_graph_count(ctx: Context) -> int:
    return int(_lib.load().fbt_graph_count(ctx.handle))


def fbt_set_mixed_tol(ctx: Context, tol: float) -> None:
    """FBT_PREC_MIXED contexts: the digit-plane tolerance (0: all planes, FP64-accurate)."""
    _check(_lib.load().fbt_set_mixed_tol(ctx.handle, float(tol)), "fbt_set_mixed_tol")


def fbt_get_mixed_tol(ctx: Context) -> float:
    return float(_lib.load().fbt_get_mixed_tol(ctx.handle))


def fbt_mixed_counts(ctx: Context, reset: bool = False) -> dict:
    """Tile-product tasks per tier since creation (or the last reset): skipped, 1, 3, 7 planes."""
    a = (C.c_longlong * 4)()
    _check(_lib.load().fbt_mixed_counts(ctx.handle, a, int(bool(reset))), "fbt_mixed_counts")
    return {"skipped": a[0], "planes1": a[1], "planes3": a[2], "planes7": a[3]}


def fbt_set_spin_budget(ctx: Context, iterations: int) -> None:
    """Test hook: iteration limit of the tensor-core kernel's waits (<= 0: the default)."""
    _check(_lib.load().fbt_set_spin_budget(ctx.handle, int(iterations)), "fbt_set_spin_budget")


def fbt_profile(ctx: Context, enable: bool) -> None:
    _check(_lib.load().fbt_profile(ctx.handle, int(bool(enable))), "fbt_profile")


def fbt_profile_read(ctx: Context) -> dict:
    lib = _lib.load()
    cnt = C.c_int()
    arr = (FbtKernelStat * 64)()
    _check(lib.fbt_profile_read(ctx.handle, arr, 64, C.byref(cnt)), "fbt_profile_read")
    return {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].ms, flops=arr[i].flops,
                                       bytes=arr[i].bytes) for i in range(min(cnt.value, 64))}


def fbt_factor_reuses(ctx: Context) -> int:
    return int(_lib.load().fbt_factor_reuses(ctx.handle))


def fbt_launch_count(ctx: Context, reset: bool = False) -> int:
    return int(_lib.load().fbt_launch_count(ctx.handle, int(bool(reset))))


def fbt_transfer_bytes(ctx: Context, reset: bool = False):
    h, d = C.c_longlong(), C.c_longlong()
    _check(_lib.load().fbt_transfer_bytes(ctx.handle, C.byref(h), C.byref(d), int(bool(reset))), "fbt_transfer_bytes")
    return h.value, d.value


def fbt_copy_slab(ctx: Context, which: int) -> np.ndarray:
    g = ctx.geometry()
    nb, T = g["nb"], g["tiles"]
    out = np.empty(T * (T + 1) // 2 * nb * nb)
    _check(_lib.load().fbt_copy_slab(ctx.handle, which, out.ctypes.data_as(C.c_void_p), 0), "fbt_copy_slab")
    return out


def fbt_copy_perm(ctx: Context) -> np.ndarray:
    out = np.empty(ctx.n, dtype=np.int64)
    _check(_lib.load().fbt_copy_perm(ctx.handle, out.ctypes.data_as(C.POINTER(C.c_longlong))), "fbt_copy_perm")
    return out


def fbt_generate(ctx: Context, theta, with_derivatives: bool = True) -> None:
    s = _lib.load().fbt_generate(ctx.handle, _dbl3(theta), int(bool(with_derivatives)))
    if s != FBT_OK:
        raise FbtError(s, "fbt_generate")


class MaternMLE:
    """Convenience wrapper: one field, Algorithm 2/3 evaluations and the Fisher-BT fit."""

    def __init__(self, locs, z, **kw):
        self.ctx = fbt_create(locs, z, **kw)

    def loglik(self, theta) -> float:
        return mle_loglik(self.ctx, theta)

    def eval(self, theta):
        return mle_eval(self.ctx, theta)

    def fit(self, theta0=None, theta_lo=None, theta_hi=None, bt=None) -> FbtState:
        return fisher_bt_run(self.ctx, theta0, theta_lo, theta_hi, bt)

    def close(self):
        fbt_destroy(self.ctx)
