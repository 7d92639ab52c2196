"""GB300-native fJOFC: Python binding of the C ABI in ``include/fjofc.h``.

The functions here only marshal arguments (torch CUDA tensors -> device pointers,
strides, the current CUDA stream) and call ``_lib/libfjofc.so``; every step of the
method runs in that library's CUDA kernels.  There is no CPU fallback: if the library
is missing or cannot be loaded, importing this package raises.

    import paper_1502_03391_gb300 as fj
    res = fj.embed(deltas, W, X, max_iter=200, tol=1e-7, tol_mode="relative")
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FJOFC_LIBRARY selects another build of the same library (e.g. a tuning variant).
LIB_PATH = os.environ.get("FJOFC_LIBRARY") or os.path.join(_HERE, "_lib", "libfjofc.so")

FJOFC_OK = 0
FJOFC_ERR_ARG = -1
FJOFC_ERR_CUDA = -2
FJOFC_ERR_NONFINITE = -3
FJOFC_ERR_TIMEOUT = -4
FJOFC_ERR_NOMEM = -5
FJOFC_ERR_UNSUPPORTED = -6

F32, F16, BF16 = 0, 1, 2
TOL_ABS_NORMALIZED, TOL_RELATIVE = 0, 1
MAX_M, MAX_D = 32, 16

# Every symbol declared in include/fjofc.h.
EXPORTS = ("fjofc_embed", "fjofc_embed_noalloc", "fjofc_stress", "fjofc_oos", "fjofc_strerror", "fjofc_version",
           "fjofc_mlp_param_count", "fjofc_mlp_init", "fjofc_mlp_features", "fjofc_mlp_forward", "fjofc_mlp_gradient",
           "fjofc_mlp_train", "fjofc_mlp_broadcast", "fjofc_mlp_select", "fjofc_plan_create", "fjofc_plan_run",
           "fjofc_plan_results", "fjofc_plan_info", "fjofc_plan_destroy", "fjofc_plan_autotune", "fjofc_init_cmds",
           "fjofc_test_barrier_skew", "fjofc_transform_rows", "fjofc_packed_size", "fjofc_pack_delta")


class FjofcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"fjofc status {status}: {message}")
        self.status = status


class _Opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("tol", ctypes.c_double), ("tol_mode", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("relax", ctypes.c_float), ("oos_form", ctypes.c_int32),
                ("check_inputs", ctypes.c_int32), ("deterministic", ctypes.c_int32),
                ("wait_limit_us", ctypes.c_int32), ("delta_layout", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("stress", ctypes.c_double),
                ("stress_normalized", ctypes.c_double), ("stress_history", ctypes.POINTER(ctypes.c_double)),
                ("ms_total", ctypes.c_float), ("passes", ctypes.c_int32), ("ms_pass", ctypes.c_float),
                ("ms_apply", ctypes.c_float), ("launches", ctypes.c_int32)]


class _Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int64), ("d", ctypes.c_int32),
                ("delta", ctypes.POINTER(ctypes.c_void_p)), ("ld", ctypes.c_int64), ("delta_dtype", ctypes.c_int32),
                ("delta_scale", ctypes.POINTER(ctypes.c_float)), ("weights", ctypes.POINTER(ctypes.c_double)),
                ("X", ctypes.c_void_p)]


class _TuneOpts(ctypes.Structure):
    _fields_ = [("probe_iters", ctypes.c_int32), ("allow_f16", ctypes.c_int32), ("reserved", ctypes.c_int32 * 6)]


class _TuneResult(ctypes.Structure):
    _fields_ = [("pass_cost", ctypes.c_float), ("barrier_cost", ctypes.c_float), ("delta_dtype", ctypes.c_int32),
                ("probe_ms", ctypes.c_float), ("candidates", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class _InitOpts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("tol", ctypes.c_double), ("reserved", ctypes.c_int32 * 4)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"fJOFC CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    lib.fjofc_embed.argtypes = [i32, i64, i32, ctypes.POINTER(vp), i64, i32, ctypes.POINTER(ctypes.c_float), dp,
                                vp, ctypes.POINTER(_Opts), ctypes.POINTER(_Result), vp]
    lib.fjofc_embed.restype = ctypes.c_int
    lib.fjofc_stress.argtypes = [i32, i64, i32, ctypes.POINTER(vp), i64, i32, ctypes.POINTER(ctypes.c_float), dp,
                                 vp, dp, vp]
    lib.fjofc_stress.restype = ctypes.c_int
    lib.fjofc_oos.argtypes = [i32, i64, i32, i64, vp, vp, i64, i32, ctypes.POINTER(ctypes.c_float), dp, vp, vp, vp,
                              ctypes.POINTER(_Opts), ctypes.POINTER(_Result), vp]
    lib.fjofc_oos.restype = ctypes.c_int
    lib.fjofc_plan_create.argtypes = [ctypes.POINTER(_Problem), i32, ctypes.POINTER(_Opts), ctypes.POINTER(vp)]
    lib.fjofc_plan_create.restype = ctypes.c_int
    lib.fjofc_plan_run.argtypes = [vp, vp]
    lib.fjofc_plan_run.restype = ctypes.c_int
    lib.fjofc_plan_results.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), dp, vp]
    lib.fjofc_plan_results.restype = ctypes.c_int
    lib.fjofc_plan_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.fjofc_plan_info.restype = ctypes.c_int
    lib.fjofc_plan_autotune.argtypes = [ctypes.POINTER(_Problem), i32, ctypes.POINTER(_Opts),
                                        ctypes.POINTER(_TuneOpts), ctypes.POINTER(vp), ctypes.POINTER(_TuneResult), vp]
    lib.fjofc_plan_autotune.restype = ctypes.c_int
    lib.fjofc_plan_destroy.argtypes = [vp]
    lib.fjofc_plan_destroy.restype = None
    lib.fjofc_init_cmds.argtypes = [i32, i64, i32, ctypes.POINTER(vp), i64, i32, ctypes.POINTER(ctypes.c_float),
                                    vp, ctypes.POINTER(_InitOpts), ctypes.POINTER(i32), vp]
    lib.fjofc_init_cmds.restype = ctypes.c_int
    lib.fjofc_transform_rows.argtypes = [i32, i64, i32, i64, i64, ctypes.POINTER(vp), i64, i32,
                                         ctypes.POINTER(ctypes.c_float), dp, vp, dp, vp, dp, vp]
    lib.fjofc_transform_rows.restype = ctypes.c_int
    lib.fjofc_packed_size.argtypes = [i64, i32, ctypes.POINTER(i64)]
    lib.fjofc_packed_size.restype = ctypes.c_int64
    lib.fjofc_pack_delta.argtypes = [i64, vp, i64, i32, vp, vp]
    lib.fjofc_pack_delta.restype = ctypes.c_int
    lib.fjofc_test_barrier_skew.argtypes = [i32]
    lib.fjofc_test_barrier_skew.restype = None
    lib.fjofc_strerror.argtypes = [ctypes.c_int]
    lib.fjofc_strerror.restype = ctypes.c_char_p
    lib.fjofc_version.argtypes = []
    lib.fjofc_version.restype = ctypes.c_char_p
    return lib


_lib = _load()


def version() -> str:
    return _lib.fjofc_version().decode()


def strerror(status: int) -> str:
    return _lib.fjofc_strerror(int(status)).decode()


def _check(status: int):
    if status != FJOFC_OK:
        raise FjofcError(status, strerror(status))


# ------------------------------------------------------------------ marshalling helpers

def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float16:
        return F16
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError(f"unsupported Delta dtype {t.dtype}")


def _stream_handle(stream, device):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


def _weights(W, m) -> np.ndarray:
    Wn = np.ascontiguousarray(np.asarray(W, dtype=np.float64))
    if Wn.shape != (m, m):
        raise ValueError(f"weights must be {m}x{m}")
    return Wn


def _scales(delta_scale, m):
    if delta_scale is None:
        return None
    arr = (ctypes.c_float * m)(*[float(v) for v in delta_scale])
    return arr


def _delta_layout(deltas: Sequence, n: int):
    """Row stride (elements) shared by all Delta matrices; each must be n x n with unit
    column stride."""
    ld = None
    code = None
    for D in deltas:
        if D.dim() != 2 or D.shape[0] != n or D.shape[1] != n or D.stride(1) != 1:
            raise ValueError("each Delta must be an n x n view with unit column stride")
        if not D.is_cuda:
            raise ValueError("Delta must be a CUDA tensor")
        c = _dtype_code(D)
        if code is None:
            code, ld = c, D.stride(0)
        elif c != code or D.stride(0) != ld:
            raise ValueError("all Delta matrices must share dtype and row stride")
    return ld, code


def padded_ld(n: int, dtype) -> int:
    """Smallest row stride >= n whose rows start on 16-byte boundaries."""
    torch = _torch()
    per = 16 // torch.tensor([], dtype=dtype).element_size()
    return (n + per - 1) // per * per


def empty_delta(n: int, dtype=None, device="cuda"):
    """An n x n CUDA matrix view whose row stride satisfies the library's alignment."""
    torch = _torch()
    dtype = dtype or torch.float32
    ld = padded_ld(n, dtype)
    buf = torch.zeros((n, ld), dtype=dtype, device=device)
    return buf[:, :n]


def to_device_delta(D: np.ndarray, dtype=None, device="cuda", scale: float = 1.0):
    """Copy a host dissimilarity matrix into an aligned CUDA view (optionally divided by
    ``scale`` before rounding to a 16-bit type)."""
    torch = _torch()
    out = empty_delta(D.shape[0], dtype, device)
    src = torch.as_tensor(np.asarray(D, dtype=np.float64) / scale)
    out.copy_(src.to(device=device, dtype=out.dtype))
    return out


# ------------------------------------------------------------------ public API

@dataclasses.dataclass
class EmbedResult:
    status: int
    iters: int
    stress: float
    stress_normalized: float
    history: Optional[np.ndarray]
    ms: float
    passes: int = 0          # profiled all-pairs passes that did work
    ms_pass: float = 0.0     # their summed device time (profile=True)
    ms_apply: float = 0.0    # summed device time of the matching W^-1 passes
    launches: int = 0        # kernels launched by the call


def embed(deltas: Sequence, weights, X, max_iter: int, tol: float = -1.0, tol_mode: str = "relative",
          delta_scale=None, stream=None, history: bool = True, check: bool = True,
          profile: int = 0, relax: float = 1.0, check_inputs: bool = False,
          wait_limit_us: int = 0, layout: str = "full", n: Optional[int] = None) -> EmbedResult:
    """In-sample fJOFC from ``X`` (in place).  ``deltas``: m CUDA n x n views (float32,
    float16 or bfloat16; row stride a multiple of 16 bytes); ``weights``: m x m;
    ``X``: contiguous float32 CUDA tensor of shape (m*n, d).  ``profile``: 0 none, 1 one
    launch per pass with per-kernel timing, 2 the persistent loop kernel timed.
    ``relax``: relaxed updates (1 = the plain Guttman transform, up to 2).
    ``check_inputs``: validate every Delta (finite, non-negative, symmetric) first.
    ``wait_limit_us``: bound of the loop's grid-wide waits (0 = 2 s).
    ``layout="packed"``: ``deltas`` are ``pack_delta`` outputs and ``n`` must be given.
    See ``fjofc_embed``."""
    m = len(deltas)
    packed = layout == "packed"
    if packed and n is None:
        raise ValueError("the packed layout needs n")
    n = int(n) if packed else int(deltas[0].shape[0])
    if X.dtype != _torch().float32 or not X.is_contiguous() or X.dim() != 2 or X.shape[0] != m * n:
        raise ValueError("X must be a contiguous float32 (m*n, d) CUDA tensor")
    d = int(X.shape[1])
    if packed:
        ld, code = int(deltas[0].shape[1]), _dtype_code(deltas[0])
    else:
        ld, code = _delta_layout(deltas, n)
    ptrs = (ctypes.c_void_p * m)(*[D.data_ptr() for D in deltas])
    Wn = _weights(weights, m)
    opts = _Opts(int(max_iter), float(tol), TOL_RELATIVE if tol_mode == "relative" else TOL_ABS_NORMALIZED,
                 int(profile), float(relax))
    opts.delta_layout = 1 if packed else 0
    opts.check_inputs = 1 if check_inputs else 0
    opts.deterministic = 1
    opts.wait_limit_us = int(wait_limit_us)
    hist = np.zeros(int(max_iter) + 1, dtype=np.float64) if history else None
    res = _Result()
    if hist is not None:
        res.stress_history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = _lib.fjofc_embed(m, n, d, ptrs, ld, code, _scales(delta_scale, m),
                          Wn.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(X.data_ptr()),
                          ctypes.byref(opts), ctypes.byref(res), _stream_handle(stream, X.device))
    if check and st not in (FJOFC_OK,):
        _check(st)
    if hist is not None:
        upto = res.iters + 1 if st in (FJOFC_OK, FJOFC_ERR_NONFINITE) else 0
        hist = hist[:upto]
    return EmbedResult(st, res.iters, res.stress, res.stress_normalized, hist, res.ms_total, res.passes,
                       res.ms_pass, res.ms_apply, res.launches)


def transform_rows(delta_rows: Sequence, weights, X, r0: int, r1: int, mu=None, delta_scale=None, stream=None):
    """One Guttman transform for objects [r0, r1) (``fjofc_transform_rows``).
    ``delta_rows``: m CUDA views of shape (r1 - r0, n) (row stride a multiple of 16 bytes
    not required); ``X``: contiguous float32 (m*n, d) CUDA tensor, the whole X_{t-1};
    ``mu``: m x d means to subtract from X_{t-1} (or None).  Returns (Xout, parts):
    Xout a float32 CUDA tensor (m, r1 - r0, d) with rows [r0, r1) of X_t, parts a float64
    numpy vector [fidelity share, commensurability share, column sums of Xout (m*d)]."""
    torch = _torch()
    m = len(delta_rows)
    n = int(delta_rows[0].shape[1])
    d = int(X.shape[1])
    if X.dtype != torch.float32 or not X.is_contiguous() or X.shape[0] != m * n:
        raise ValueError("X must be a contiguous float32 (m*n, d) CUDA tensor")
    for D in delta_rows:
        if tuple(D.shape) != (r1 - r0, n) or D.stride(1) != 1:
            raise ValueError("delta_rows[l] must be a (r1 - r0, n) view with unit column stride")
    ld = int(delta_rows[0].stride(0)) if r1 - r0 > 1 else n
    code = _dtype_code(delta_rows[0])
    ptrs = (ctypes.c_void_p * m)(*[D.data_ptr() for D in delta_rows])
    Wn = _weights(weights, m)
    Xout = torch.empty((m, r1 - r0, d), dtype=torch.float32, device=X.device)
    parts = np.zeros(2 + m * d, dtype=np.float64)
    mu_arr = None if mu is None else np.ascontiguousarray(np.asarray(mu, dtype=np.float64).reshape(m * d))
    dp = ctypes.POINTER(ctypes.c_double)
    st = _lib.fjofc_transform_rows(m, n, d, int(r0), int(r1), ptrs, ld, code, _scales(delta_scale, m),
                                   Wn.ctypes.data_as(dp), ctypes.c_void_p(X.data_ptr()),
                                   None if mu_arr is None else mu_arr.ctypes.data_as(dp),
                                   ctypes.c_void_p(Xout.data_ptr()), parts.ctypes.data_as(dp),
                                   _stream_handle(stream, X.device))
    _check(st)
    return Xout, parts


def pack_delta(D, stream=None):
    """The packed band layout of a symmetric CUDA n x n matrix view (``fjofc_pack_delta``):
    returns a 2-D CUDA tensor (packed rows, ld) to pass to ``embed(..., layout="packed")``."""
    torch = _torch()
    n = int(D.shape[0])
    code = _dtype_code(D)
    ld = ctypes.c_int64(0)
    size = _lib.fjofc_packed_size(n, code, ctypes.byref(ld))
    if size < 0:
        raise ValueError("invalid size or type")
    out = torch.empty(int(size), dtype=D.dtype, device=D.device).reshape(-1, ld.value)
    _check(_lib.fjofc_pack_delta(n, ctypes.c_void_p(D.data_ptr()), int(D.stride(0)), code,
                                 ctypes.c_void_p(out.data_ptr()), _stream_handle(stream, D.device)))
    return out


def test_barrier_skew(extra: int) -> None:
    """Test support: the next in-sample loop's first grid-wide wait expects ``extra``
    arrivals more than its CTAs make (``fjofc_test_barrier_skew``)."""
    _lib.fjofc_test_barrier_skew(int(extra))


def stress(deltas: Sequence, weights, X, delta_scale=None, stream=None) -> float:
    """Raw stress sigma(X) (Eq. stress) through the library's all-pairs pass."""
    m = len(deltas)
    n = int(deltas[0].shape[0])
    d = int(X.shape[1])
    ld, code = _delta_layout(deltas, n)
    ptrs = (ctypes.c_void_p * m)(*[D.data_ptr() for D in deltas])
    Wn = _weights(weights, m)
    out = ctypes.c_double(0.0)
    st = _lib.fjofc_stress(m, n, d, ptrs, ld, code, _scales(delta_scale, m),
                           Wn.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(X.data_ptr()),
                           ctypes.byref(out), _stream_handle(stream, X.device))
    _check(st)
    return out.value


def init_cmds(deltas: Sequence, d: int, X=None, max_iter: int = 0, tol: float = 0.0, delta_scale=None,
              stream=None):
    """Algorithm 2's initial configuration X_(0) (classical MDS of the average and of
    every Delta_i, Procrustes onto the average's); see ``fjofc_init_cmds``.  ``X``: a
    contiguous float32 (m*n, d) CUDA tensor to write (allocated if None).  Returns
    ``(X, iters)`` with the subspace iterations of the m + 1 eigenproblems."""
    torch = _torch()
    m = len(deltas)
    n = int(deltas[0].shape[0])
    ld, code = _delta_layout(deltas, n)
    if X is None:
        X = torch.empty((m * n, d), dtype=torch.float32, device=deltas[0].device)
    if X.dtype != torch.float32 or not X.is_contiguous() or X.dim() != 2 or X.shape != (m * n, d):
        raise ValueError("X must be a contiguous float32 (m*n, d) CUDA tensor")
    ptrs = (ctypes.c_void_p * m)(*[D.data_ptr() for D in deltas])
    opts = _InitOpts(int(max_iter), float(tol))
    iters = (ctypes.c_int32 * (m + 1))()
    st = _lib.fjofc_init_cmds(m, n, d, ptrs, ld, code, _scales(delta_scale, m), ctypes.c_void_p(X.data_ptr()),
                              ctypes.byref(opts), iters, _stream_handle(stream, X.device))
    _check(st)
    return X, [int(v) for v in iters]


@dataclasses.dataclass
class OOSResult:
    status: int
    max_iters: int
    stress_sum: float
    ms: float


_OOS_FORMS = {"auto": 0, "streaming": 1, "resident": 2}


def oos(X, delta_new, weights, Y, max_iter: int, tol: float = -1.0, tol_mode: str = "relative",
        iters_out=None, stress_out=None, delta_scale=None, stream=None, check: bool = True,
        form: str = "auto") -> OOSResult:
    """Out-of-sample embedding of k new objects (in place in ``Y``).  ``X``: float32 CUDA
    (m*n, d) in-sample configuration; ``delta_new``: CUDA (k, m, n) view with unit stride in
    the last dimension, row stride ``ld`` = stride(1), stride(0) = m*ld; ``Y``: contiguous
    float32 CUDA (k, m, d).  ``iters_out`` (int32 [k]) and ``stress_out`` (float64 [k]) are
    optional CUDA outputs.  ``form``: "auto", "streaming" or "resident" (``fjofc_opts.oos_form``)."""
    torch = _torch()
    k, m, n = (int(s) for s in delta_new.shape)
    d = int(X.shape[1])
    if delta_new.stride(2) != 1 or delta_new.stride(0) != m * delta_new.stride(1):
        raise ValueError("delta_new must be a (k, m, n) view over a (k, m, ld) buffer")
    if not (Y.is_contiguous() and Y.dtype == torch.float32 and tuple(Y.shape) == (k, m, d)):
        raise ValueError("Y must be a contiguous float32 (k, m, d) tensor")
    if not (X.is_contiguous() and X.dtype == torch.float32 and tuple(X.shape) == (m * n, d)):
        raise ValueError("X must be a contiguous float32 (m*n, d) tensor")
    ld = delta_new.stride(1)
    code = _dtype_code(delta_new)
    Wn = _weights(weights, m)
    opts = _Opts(int(max_iter), float(tol), TOL_RELATIVE if tol_mode == "relative" else TOL_ABS_NORMALIZED)
    opts.oos_form = _OOS_FORMS[form]
    res = _Result()
    ip = ctypes.c_void_p(iters_out.data_ptr()) if iters_out is not None else None
    sp = ctypes.c_void_p(stress_out.data_ptr()) if stress_out is not None else None
    st = _lib.fjofc_oos(m, n, d, k, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(delta_new.data_ptr()), ld, code,
                        _scales(delta_scale, m), Wn.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        ctypes.c_void_p(Y.data_ptr()), ip, sp, ctypes.byref(opts), ctypes.byref(res),
                        _stream_handle(stream, X.device))
    if check:
        _check(st)
    return OOSResult(st, res.iters, res.stress, res.ms_total)


def empty_oos_delta(k: int, m: int, n: int, dtype=None, device="cuda"):
    """A (k, m, n) CUDA view whose rows satisfy the library's 16-byte alignment."""
    torch = _torch()
    dtype = dtype or torch.float32
    ld = padded_ld(n, dtype)
    buf = torch.zeros((k, m, ld), dtype=dtype, device=device)
    return buf[:, :, :n]


# ------------------------------------------------------------------ batched plans

@dataclasses.dataclass
class PlanResults:
    status: np.ndarray
    iters: np.ndarray
    stress: np.ndarray


class Plan:
    """Many independent in-sample problems run together (``fjofc_plan_*``).  ``problems``
    is a sequence of (deltas, weights, X) or (deltas, weights, X, delta_scale) with the
    same conventions as ``embed``; every problem gets the same loop options."""

    def __init__(self, problems, max_iter: int, tol: float = -1.0, tol_mode: str = "relative",
                 autotune: bool = False, probe_iters: int = 8, allow_f16: bool = False, stream=None,
                 layout: str = "full", n=None):
        """``autotune``: let ``fjofc_plan_autotune`` time candidate schedules (and float16
        storage of float32 Delta when ``allow_f16``) on ``probe_iters`` transforms and keep
        the fastest; the choice is in ``self.tuning``.  ``layout="packed"``: every Delta is
        a ``pack_delta`` output and ``n`` lists the problems' object counts."""
        keep = []
        packed = layout == "packed"
        arr = (_Problem * len(problems))()
        for i, pr in enumerate(problems):
            deltas, W, X = pr[0], pr[1], pr[2]
            scale = pr[3] if len(pr) > 3 else None
            m = len(deltas)
            if packed:
                n_i = int(n[i])
                ld, code = int(deltas[0].shape[1]), _dtype_code(deltas[0])
            else:
                n_i = int(deltas[0].shape[0])
                ld, code = _delta_layout(deltas, n_i)
            ptrs = (ctypes.c_void_p * m)(*[D.data_ptr() for D in deltas])
            Wn = _weights(W, m)
            sc = _scales(scale, m)
            keep += [ptrs, Wn, sc]
            arr[i] = _Problem(m, n_i, int(X.shape[1]), ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p)), ld, code,
                              ctypes.cast(sc, ctypes.POINTER(ctypes.c_float)) if sc is not None else None,
                              Wn.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(X.data_ptr()))
        opts = _Opts(int(max_iter), float(tol), TOL_RELATIVE if tol_mode == "relative" else TOL_ABS_NORMALIZED)
        opts.delta_layout = 1 if packed else 0
        h = ctypes.c_void_p()
        self.tuning = None
        if autotune:
            torch = _torch()
            to = _TuneOpts(int(probe_iters), 1 if allow_f16 else 0)
            tr = _TuneResult()
            _check(_lib.fjofc_plan_autotune(arr, len(problems), ctypes.byref(opts), ctypes.byref(to), ctypes.byref(h),
                                            ctypes.byref(tr), _stream_handle(stream, torch.device("cuda"))))
            self.tuning = {"pass_cost": tr.pass_cost, "barrier_cost": tr.barrier_cost,
                           "float16_delta": tr.delta_dtype == F16, "probe_ms": tr.probe_ms,
                           "candidates": tr.candidates}
        else:
            _check(_lib.fjofc_plan_create(arr, len(problems), ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        self.count = len(problems)

    def run(self, stream=None):
        torch = _torch()
        _check(_lib.fjofc_plan_run(self._h, _stream_handle(stream, torch.device("cuda"))))

    def results(self, stream=None, check: bool = True) -> PlanResults:
        torch = _torch()
        st = (ctypes.c_int32 * self.count)()
        it = (ctypes.c_int32 * self.count)()
        sg = (ctypes.c_double * self.count)()
        rc = _lib.fjofc_plan_results(self._h, st, it, sg, _stream_handle(stream, torch.device("cuda")))
        if check:
            _check(rc)
        return PlanResults(np.array(st[:]), np.array(it[:]), np.array(sg[:]))

    def info(self):
        g = (ctypes.c_int32 * self.count)()
        graphed = ctypes.c_int32(0)
        launches = ctypes.c_int32(0)
        _check(_lib.fjofc_plan_info(self._h, g, ctypes.byref(graphed), ctypes.byref(launches)))
        return {"groups": np.array(g[:]), "graphed": bool(graphed.value), "launches": launches.value}

    def close(self):
        if getattr(self, "_h", None):
            _lib.fjofc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
