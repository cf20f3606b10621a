"""Thin ctypes binding of the C ABI in ``include/qoc.h`` (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libqoc.so``; this module converts numpy
arrays to the interleaved complex128 layout the ABI expects and turns status codes into
exceptions.  There is no CPU fallback: if the library is missing or cannot be loaded, every
entry point raises ``QocError``.

The module-level functions carry the names of the C entry points (``qoc_create``,
``qoc_set_system``, ...); ``Context`` wraps them for convenience, and ``QOCCost`` is a
``torch.autograd.Function`` over ``qoc_evaluate_device``.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libqoc.so")

QOC_OK = 0
STATUS_NAMES = {0: "QOC_OK", 1: "QOC_ERR_ARG", 2: "QOC_ERR_SHAPE", 3: "QOC_ERR_NOT_HERMITIAN",
                4: "QOC_ERR_NONFINITE", 5: "QOC_ERR_STATE", 6: "QOC_ERR_OOM", 7: "QOC_ERR_CUDA",
                8: "QOC_ERR_TIMEOUT", 9: "QOC_ERR_UNSUPPORTED", 10: "QOC_ERR_RANGE", 11: "QOC_ERR_STALE"}
PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
SWEEPS = {"auto": 0, "serial": 1, "scan": 2}
GRADIENTS = {"exact": 0, "first_order": 1}
ADJOINTS = {"auto": 0, "recompute": 1}
PROPAGATIONS = {"unitary": 0, "state": 1}
EXPONENTIALS = {"taylor": 0, "chebyshev": 1}
TAYLOR_SCHEMES = {"auto": 0, "horner": 1}

# every symbol exported by include/qoc.h
ABI_SYMBOLS = ("qoc_default_options", "qoc_create", "qoc_destroy", "qoc_last_error", "qoc_status_string",
               "qoc_set_system", "qoc_set_targets", "qoc_set_ensemble", "qoc_evaluate_cost_and_grad",
               "qoc_evaluate_device", "qoc_sync", "qoc_get_info", "qoc_get_profile", "qoc_reset_profile",
               "qoc_evaluate_static", "qoc_evaluate_batch", "qoc_batch_create", "qoc_batch_launch",
               "qoc_batch_sync", "qoc_batch_destroy", "qoc_measure_fma_peak")


class QocError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class qoc_options(ct.Structure):
    _fields_ = [("precision", ct.c_int), ("tol", ct.c_double), ("theta_max", ct.c_double),
                ("ckpt_stride", ct.c_int), ("device", ct.c_int), ("stream", ct.c_void_p),
                ("p_override", ct.c_int), ("n_override", ct.c_int), ("profile", ct.c_int),
                ("wave_slices", ct.c_int), ("plain_fp32_exp", ct.c_int), ("sweep", ct.c_int),
                ("gradient", ct.c_int), ("adjoint", ct.c_int), ("graph", ct.c_int), ("fault_inject", ct.c_int),
                ("reversal", ct.c_int), ("propagation", ct.c_int), ("exponential", ct.c_int),
                ("taylor_scheme", ct.c_int), ("autotune", ct.c_int)]


PROFILE_SLOTS = 16


class qoc_profile(ct.Structure):
    _fields_ = [("count", ct.c_int), ("name", (ct.c_char * 32) * PROFILE_SLOTS),
                ("launches", ct.c_longlong * PROFILE_SLOTS), ("total_ms", ct.c_double * PROFILE_SLOTS)]


class qoc_info(ct.Structure):
    _fields_ = [("p", ct.c_int), ("n", ct.c_int), ("theta", ct.c_double), ("ckpt_stride", ct.c_int),
                ("wave_slices", ct.c_int), ("n_waves", ct.c_int), ("launches_per_eval", ct.c_int), ("kernel_path", ct.c_int),
                ("device_bytes", ct.c_longlong), ("adjoint_form", ct.c_int), ("taylor_scheme", ct.c_int),
                ("autotune_candidates", ct.c_int)]


_lib = None


def load(path: str = LIB_PATH) -> ct.CDLL:
    """Loads the CUDA library (once).  Raises QocError if it is absent: no fallback exists."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise QocError(7, f"CUDA library not built: {path} (run paper_1612_04929_gb300.build)")
    lib = ct.CDLL(path)
    P, I, D, VP = ct.c_void_p, ct.c_int, ct.c_double, ct.c_void_p
    DP = ct.POINTER(ct.c_double)
    lib.qoc_default_options.argtypes = [ct.POINTER(qoc_options)]
    lib.qoc_default_options.restype = None
    lib.qoc_create.argtypes = [ct.POINTER(P), ct.POINTER(qoc_options)]
    lib.qoc_create.restype = I
    lib.qoc_destroy.argtypes = [P]
    lib.qoc_destroy.restype = None
    lib.qoc_last_error.argtypes = [P]
    lib.qoc_last_error.restype = ct.c_char_p
    lib.qoc_status_string.argtypes = [I]
    lib.qoc_status_string.restype = ct.c_char_p
    lib.qoc_set_system.argtypes = [P, I, I, DP, DP, D, I]
    lib.qoc_set_system.restype = I
    lib.qoc_set_targets.argtypes = [P, I, DP, DP, I, ct.POINTER(ct.c_int), DP, DP, DP]
    lib.qoc_set_targets.restype = I
    lib.qoc_set_ensemble.argtypes = [P, I, DP, DP]
    lib.qoc_set_ensemble.restype = I
    lib.qoc_evaluate_cost_and_grad.argtypes = [P, DP, DP, DP, DP]
    lib.qoc_evaluate_cost_and_grad.restype = I
    lib.qoc_evaluate_device.argtypes = [P, VP, VP, VP]
    lib.qoc_evaluate_device.restype = I
    lib.qoc_sync.argtypes = [P]
    lib.qoc_sync.restype = I
    lib.qoc_get_info.argtypes = [P, ct.POINTER(qoc_info)]
    lib.qoc_get_info.restype = I
    lib.qoc_get_profile.argtypes = [P, ct.POINTER(qoc_profile)]
    lib.qoc_get_profile.restype = I
    lib.qoc_reset_profile.argtypes = [P]
    lib.qoc_reset_profile.restype = I
    lib.qoc_evaluate_static.argtypes = [I, I, I, I, D, VP, VP, VP, VP, VP, VP, DP, VP, VP, VP]
    lib.qoc_evaluate_static.restype = I
    PP = ct.POINTER(ct.c_void_p)
    lib.qoc_evaluate_batch.argtypes = [I, PP, PP, PP, PP, VP]
    lib.qoc_evaluate_batch.restype = I
    lib.qoc_batch_create.argtypes = [I, PP, PP, PP, PP, VP, ct.POINTER(P)]
    lib.qoc_batch_create.restype = I
    lib.qoc_batch_launch.argtypes = [P, VP]
    lib.qoc_batch_launch.restype = I
    lib.qoc_batch_sync.argtypes = [P]
    lib.qoc_batch_sync.restype = I
    lib.qoc_batch_destroy.argtypes = [P]
    lib.qoc_batch_destroy.restype = None
    lib.qoc_measure_fma_peak.argtypes = [I, I, DP, ct.POINTER(ct.c_int)]
    lib.qoc_measure_fma_peak.restype = I
    _lib = lib
    return lib


def _dp(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ct.POINTER(ct.c_double))


def _c128(a, shape=None) -> np.ndarray:
    """complex array -> contiguous complex128 (viewed as interleaved doubles by the ABI)."""
    x = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if shape is not None and x.shape != tuple(shape):
        x = x.reshape(shape)
    return x


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(ctx, status: int):
    if status != QOC_OK:
        msg = load().qoc_last_error(ctx).decode() if ctx else ""
        raise QocError(status, msg)


# ------------------------------------------------------------------ C-named entry points
def qoc_default_options() -> qoc_options:
    o = qoc_options()
    load().qoc_default_options(ct.byref(o))
    return o


def qoc_create(opt: Optional[qoc_options] = None) -> ct.c_void_p:
    ctx = ct.c_void_p()
    st = load().qoc_create(ct.byref(ctx), ct.byref(opt) if opt is not None else None)
    if st != QOC_OK:
        raise QocError(st, "qoc_create failed")
    return ctx


def qoc_destroy(ctx) -> None:
    load().qoc_destroy(ctx)


def qoc_last_error(ctx) -> str:
    return load().qoc_last_error(ctx).decode()


def qoc_status_string(status: int) -> str:
    return load().qoc_status_string(status).decode()


def qoc_set_system(ctx, H0, Hk, dt: float, N: int) -> None:
    H0 = _c128(H0)
    d = H0.shape[0]
    Hk = _c128(Hk).reshape(-1, d, d) if Hk is not None and np.size(Hk) else np.zeros((0, d, d), np.complex128)
    M = Hk.shape[0]
    _check(ctx, load().qoc_set_system(ctx, d, M, _dp(H0.view(np.float64)),
                                      _dp(Hk.view(np.float64)) if M else None, float(dt), int(N)))


def qoc_set_targets(ctx, psi0, psiT, forbidden: Sequence[int] = (), col_weight=None, psiT_path=None,
                    alpha=(1.0, 0, 0, 0, 0)) -> None:
    psi0 = _c128(psi0)
    if psi0.ndim == 1:
        psi0 = psi0[:, None].copy()
    d, S = psi0.shape
    psiT = _c128(psiT).reshape(d, S)
    forb = np.ascontiguousarray(np.asarray(forbidden, dtype=np.int32))
    w = None if col_weight is None else _f64(col_weight)
    path = None if psiT_path is None else _c128(psiT_path)
    al = _f64(alpha)
    _check(ctx, load().qoc_set_targets(
        ctx, S, _dp(psi0.view(np.float64)), _dp(psiT.view(np.float64)), len(forb),
        forb.ctypes.data_as(ct.POINTER(ct.c_int)) if len(forb) else None, _dp(w),
        _dp(path.view(np.float64)) if path is not None else None, _dp(al)))


def qoc_set_ensemble(ctx, delta, Hdet=None) -> None:
    delta = _f64(delta).reshape(-1)
    Hd = None if Hdet is None else _c128(Hdet)
    _check(ctx, load().qoc_set_ensemble(ctx, len(delta), _dp(delta),
                                        _dp(Hd.view(np.float64)) if Hd is not None else None))


def qoc_evaluate_cost_and_grad(ctx, u, M: int, N: int):
    u = _f64(u).reshape(M, N)
    grad = np.zeros((M, N), np.float64)
    cost = ct.c_double()
    terms = np.zeros(5, np.float64)
    _check(ctx, load().qoc_evaluate_cost_and_grad(ctx, _dp(u), ct.byref(cost), _dp(grad), _dp(terms)))
    return cost.value, grad, terms


def qoc_evaluate_device(ctx, u_dev: int, grad_dev: int, out_dev: int) -> None:
    _check(ctx, load().qoc_evaluate_device(ctx, ct.c_void_p(u_dev), ct.c_void_p(grad_dev), ct.c_void_p(out_dev)))


def qoc_sync(ctx) -> None:
    _check(ctx, load().qoc_sync(ctx))


def qoc_get_info(ctx) -> dict:
    info = qoc_info()
    _check(ctx, load().qoc_get_info(ctx, ct.byref(info)))
    return {f: getattr(info, f) for f, _ in qoc_info._fields_}


def qoc_get_profile(ctx) -> dict:
    """{kernel class: (launches, total_ms)} accumulated since the last reset."""
    pr = qoc_profile()
    _check(ctx, load().qoc_get_profile(ctx, ct.byref(pr)))
    return {pr.name[i].value.decode(): (pr.launches[i], pr.total_ms[i]) for i in range(pr.count)}


def qoc_reset_profile(ctx) -> None:
    _check(ctx, load().qoc_reset_profile(ctx))


def qoc_evaluate_static(d: int, M: int, N: int, S: int, dt: float, H0_dev: int, Hk_dev: int, u_dev: int,
                        psi0_dev: int, psiT_dev: int, fmask_dev: int, alpha, grad_dev: int, out_dev: int,
                        stream: int = 0) -> None:
    """The evaluation that allocates no memory (see include/qoc.h): every array argument except
    ``alpha`` is a raw device pointer (int); the call is asynchronous on ``stream``."""
    al = _f64(alpha)
    st = load().qoc_evaluate_static(d, M, N, S, float(dt), H0_dev or None, Hk_dev or None, u_dev or None,
                                    psi0_dev or None, psiT_dev or None, fmask_dev or None, _dp(al),
                                    grad_dev or None, out_dev or None, stream or None)
    if st != QOC_OK:
        raise QocError(st, "qoc_evaluate_static failed")


def qoc_evaluate_batch(ctxs, u_dev, grad_dev, out_dev, stream: int = 0) -> None:
    """Batched evaluation (see include/qoc.h): ``ctxs`` are Context objects or raw handles, the
    other lists raw device pointers (ints), one per problem."""
    n = len(ctxs)
    arr = lambda xs: (ct.c_void_p * n)(*[ct.c_void_p(int(x)) for x in xs])
    handles = (ct.c_void_p * n)(*[(c.handle if isinstance(c, Context) else c) for c in ctxs])
    st = load().qoc_evaluate_batch(n, handles, arr(u_dev), arr(grad_dev), arr(out_dev), stream or None)
    if st != QOC_OK:
        msgs = [load().qoc_last_error(c.handle if isinstance(c, Context) else c).decode() for c in ctxs]
        raise QocError(st, "; ".join(m for m in msgs if m))


def _batch_errors(ctxs):
    return "; ".join(m for m in (load().qoc_last_error(c.handle if isinstance(c, Context) else c).decode()
                                 for c in ctxs) if m)


class Batch:
    """A batch captured into one CUDA graph (qoc_batch_create, see include/qoc.h): ``ctxs`` are
    Context objects or raw handles, the other lists raw device pointers, one per problem.
    Creating it evaluates the batch once (synchronising ``stream``); ``launch`` replays the
    graph, ``sync`` waits and raises on a device-side error (QOC_ERR_STALE when the controls
    outgrew the frozen orders).  Close the batch before its contexts."""

    def __init__(self, ctxs, u_dev, grad_dev, out_dev, stream: int = 0):
        n = len(ctxs)
        arr = lambda xs: (ct.c_void_p * n)(*[ct.c_void_p(int(x)) for x in xs])
        handles = (ct.c_void_p * n)(*[(c.handle if isinstance(c, Context) else c) for c in ctxs])
        self._ctxs = list(ctxs)
        b = ct.c_void_p()
        st = load().qoc_batch_create(n, handles, arr(u_dev), arr(grad_dev), arr(out_dev), stream or None,
                                     ct.byref(b))
        if st != QOC_OK:
            raise QocError(st, _batch_errors(self._ctxs))
        self._b = b.value
        for c in self._ctxs:
            if isinstance(c, Context):
                c._batches += 1

    def launch(self, stream: int = 0):
        st = load().qoc_batch_launch(self._b, stream or None)
        if st != QOC_OK:
            raise QocError(st, _batch_errors(self._ctxs))

    def sync(self):
        st = load().qoc_batch_sync(self._b)
        if st != QOC_OK:
            raise QocError(st, _batch_errors(self._ctxs))

    def close(self):
        if getattr(self, "_b", None):
            load().qoc_batch_destroy(self._b)
            self._b = None
            for c in self._ctxs:
                if isinstance(c, Context):
                    c._batches -= 1

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def qoc_measure_fma_peak(device: int = 0, fp64: bool = False):
    """Measured FP32 (or FP64) multiply-add throughput of the device in TFLOP/s and its SM count
    (see include/qoc.h)."""
    t = ct.c_double(0.0)
    n = ct.c_int(0)
    st = load().qoc_measure_fma_peak(int(device), 1 if fp64 else 0, ct.byref(t), ct.byref(n))
    if st != QOC_OK:
        raise QocError(st, "qoc_measure_fma_peak failed")
    return t.value, n.value


# ------------------------------------------------------------------ convenience wrapper
class Context:
    """One evaluation context (owns device memory and a CUDA stream)."""

    def __init__(self, precision: str = "fp64", *, tol: float = 0.0, theta_max: float = 0.0,
                 ckpt_stride: int = 0, wave_slices: int = 0, device: int = 0, stream: Optional[int] = None,
                 p_override: int = 0, n_override: int = -1, profile: bool = False,
                 plain_fp32_exp: bool = False, sweep: str = "auto", gradient: str = "exact",
                 adjoint: str = "auto", graph: bool = False, fault_inject: int = 0, reversal: bool = False,
                 propagation: str = "unitary", exponential: str = "taylor", taylor_scheme: str = "auto",
                 autotune: bool = False):
        opt = qoc_default_options()
        opt.precision = PRECISIONS[precision]
        opt.tol = tol
        opt.theta_max = theta_max
        opt.ckpt_stride = ckpt_stride
        opt.wave_slices = wave_slices
        opt.device = device
        # stream=None: the context owns a stream; 0 (torch's default stream) maps to the legacy
        # default stream handle so that kernels and torch work are ordered on the same stream
        opt.stream = None if stream is None else (stream if stream != 0 else 1)
        opt.p_override = p_override
        opt.n_override = n_override
        opt.profile = 1 if profile else 0
        opt.plain_fp32_exp = 1 if plain_fp32_exp else 0
        opt.sweep = SWEEPS[sweep]
        opt.gradient = GRADIENTS[gradient]
        opt.adjoint = ADJOINTS[adjoint]
        opt.graph = 1 if graph else 0
        opt.fault_inject = fault_inject
        opt.reversal = 1 if reversal else 0
        opt.propagation = PROPAGATIONS[propagation]
        opt.exponential = EXPONENTIALS[exponential]
        opt.taylor_scheme = TAYLOR_SCHEMES[taylor_scheme]
        opt.autotune = 1 if autotune else 0
        self.precision = precision
        self._batches = 0
        self._ctx = qoc_create(opt)
        self.M = self.N = 0

    def close(self):
        if getattr(self, "_ctx", None):
            if self._batches:
                raise QocError(5, "the context belongs to a captured batch: close the batch first")
            qoc_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._ctx

    def set_system(self, H0, Hk, dt, N):
        qoc_set_system(self._ctx, H0, Hk, dt, N)
        H0 = np.asarray(H0)
        self.M = 0 if Hk is None else int(np.asarray(Hk).reshape(-1, H0.shape[0], H0.shape[0]).shape[0])
        self.N = int(N)

    def set_targets(self, psi0, psiT, forbidden=(), col_weight=None, psiT_path=None, alpha=(1.0, 0, 0, 0, 0)):
        qoc_set_targets(self._ctx, psi0, psiT, forbidden, col_weight, psiT_path, alpha)

    def set_ensemble(self, delta, Hdet=None):
        qoc_set_ensemble(self._ctx, delta, Hdet)

    def set_problem(self, prob):
        """Loads a ``synthetic.Problem``-like object (H0, Hk, dt, N, psi0, psiT, forbidden,
        col_weight, psiT_path, alpha, delta, Hdet)."""
        self.set_system(prob.H0, prob.Hk, prob.dt, prob.N)
        self.set_targets(prob.psi0, prob.psiT, prob.forbidden, prob.col_weight, prob.psiT_path, prob.alpha)
        if len(prob.delta) > 1 or np.any(prob.delta != 0):
            self.set_ensemble(prob.delta, prob.Hdet)

    def evaluate(self, u):
        """(cost, grad (M, N), terms (5,)) from host memory."""
        u = np.atleast_2d(np.asarray(u, np.float64))
        M, N = (self.M, self.N) if self.N else u.shape
        return qoc_evaluate_cost_and_grad(self._ctx, u, M, N)

    def evaluate_device(self, u_dev: int, grad_dev: int, out_dev: int):
        qoc_evaluate_device(self._ctx, u_dev, grad_dev, out_dev)

    def sync(self):
        qoc_sync(self._ctx)

    def info(self) -> dict:
        return qoc_get_info(self._ctx)

    def profile(self) -> dict:
        return qoc_get_profile(self._ctx)

    def reset_profile(self):
        qoc_reset_profile(self._ctx)

    def evaluate_host_ptr(self, u_ptr: int, grad_ptr: int):
        """Host-API evaluation on raw host pointers (e.g. pinned buffers): returns (cost, terms)."""
        cost = ct.c_double()
        terms = np.zeros(5, np.float64)
        _check(self._ctx, load().qoc_evaluate_cost_and_grad(
            self._ctx, ct.cast(ct.c_void_p(u_ptr), ct.POINTER(ct.c_double)), ct.byref(cost),
            ct.cast(ct.c_void_p(grad_ptr), ct.POINTER(ct.c_double)), _dp(terms)))
        return cost.value, terms


def _make_autograd():
    import torch

    class QOCCost(torch.autograd.Function):
        """C(u) with dC/du from the hand-written adjoint: forward runs qoc_evaluate_device on
        the context stream (which must be torch's current stream) and keeps the gradient;
        backward scales it by the incoming gradient."""

        @staticmethod
        def forward(fctx, qctx: Context, u):
            if not (u.is_cuda and u.dtype == torch.float64 and u.is_contiguous()):
                raise QocError(1, "u must be a contiguous float64 CUDA tensor")
            grad = torch.empty_like(u)
            out = torch.empty(6, dtype=torch.float64, device=u.device)
            qctx.evaluate_device(u.data_ptr(), grad.data_ptr(), out.data_ptr())
            fctx.save_for_backward(grad)
            fctx.mark_non_differentiable(out)
            return out[0], out[1:]

        @staticmethod
        def backward(fctx, gcost, gterms):
            (grad,) = fctx.saved_tensors
            return None, grad * gcost

    return QOCCost


_QOCCost = None


def QOCCost():
    """The torch.autograd.Function class (created on first use, so that importing this module
    does not import torch)."""
    global _QOCCost
    if _QOCCost is None:
        _QOCCost = _make_autograd()
    return _QOCCost


def cost(qctx: Context, u):
    """Differentiable total cost C(u) of a CUDA float64 tensor u (M, N); returns (C, terms)."""
    return QOCCost().apply(qctx, u)
