"""Host-side checks of the C-ABI library (no GPU needed).

The shared library must load on a machine without a GPU, export every function that
``include/fjofc.h`` declares, and reject invalid arguments before it touches CUDA
(argument validation precedes any runtime call, so dummy device pointers are safe).
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fjofc.h")


def _lib():
    from conftest import ensure_library
    return ensure_library()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fjofc_[a-z_]+)\s*\(", src)))


def test_header_declares_expected_api():
    assert _declared_functions() == sorted(["fjofc_embed", "fjofc_embed_noalloc", "fjofc_stress", "fjofc_oos",
                                            "fjofc_strerror", "fjofc_version", "fjofc_mlp_param_count",
                                            "fjofc_mlp_init", "fjofc_mlp_features", "fjofc_mlp_forward",
                                            "fjofc_mlp_gradient", "fjofc_mlp_train", "fjofc_mlp_broadcast",
                                            "fjofc_mlp_select", "fjofc_plan_create", "fjofc_plan_run",
                                            "fjofc_plan_results", "fjofc_plan_info", "fjofc_plan_destroy",
                                            "fjofc_plan_autotune", "fjofc_init_cmds", "fjofc_test_barrier_skew",
                                            "fjofc_transform_rows", "fjofc_packed_size", "fjofc_pack_delta"])


def test_library_loads_and_exports_every_declared_symbol():
    fj = _lib()
    raw = ctypes.CDLL(fj.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(raw, name), name
    assert set(fj.EXPORTS) == set(_declared_functions())
    assert "sm_103a" in fj.version()
    assert fj.strerror(0) == "ok"


# ------------------------------------------------------------------ argument validation

class _Call:
    """Calls fjofc_embed with dummy (never dereferenced) device pointers."""

    def __init__(self, fj):
        self.fj = fj
        self.lib = ctypes.CDLL(fj.LIB_PATH)
        self.lib.fjofc_embed.restype = ctypes.c_int

    def embed(self, m=2, n=8, d=2, ld=8, dtype=0, W=None, ptr=4096, X=8192, max_iter=5, tol_mode=1,
              scales=None, relax=0.0, **fields):
        fj = self.fj
        W = np.array([[1.0, 0.5], [0.5, 1.0]]) if W is None else np.asarray(W, dtype=np.float64)
        ptrs = (ctypes.c_void_p * max(m, 1))(*([ptr] * max(m, 1)))
        opts = fj._Opts(max_iter, -1.0, tol_mode, 0, relax)
        for k, v in fields.items():
            if k == "reserved":
                opts.reserved[0] = v
            else:
                setattr(opts, k, v)
        sc = None if scales is None else (ctypes.c_float * m)(*scales)
        return self.lib.fjofc_embed(ctypes.c_int32(m), ctypes.c_int64(n), ctypes.c_int32(d), ptrs,
                                    ctypes.c_int64(ld), ctypes.c_int32(dtype), sc,
                                    W.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(X),
                                    ctypes.byref(opts), None, None)


@pytest.fixture(scope="module")
def call():
    return _Call(_lib())


@pytest.mark.parametrize("kw,code", [
    (dict(m=0), -1),
    (dict(m=33, W=np.eye(33)), -6),      # beyond FJOFC_MAX_M = 32
    (dict(n=1, ld=4), -1),
    (dict(d=0), -1),
    (dict(d=17), -6),
    (dict(n=5, ld=6), -1),                  # 24-byte rows are not 16-byte aligned
    (dict(ld=4), -1),                       # ld < n
    (dict(ptr=4100), -1),                   # misaligned Delta base
    (dict(X=0), -1),
    (dict(max_iter=-1), -1),
    (dict(tol_mode=7), -1),
    (dict(dtype=5), -1),
    (dict(W=[[1.0, 0.5], [0.4, 1.0]]), -1),  # asymmetric
    (dict(W=[[0.0, 0.5], [0.5, 1.0]]), -1),  # w_ii must be > 0
    (dict(W=[[1.0, -0.5], [-0.5, 1.0]]), -1),  # w_ij must be >= 0
    (dict(W=[[np.nan, 0.5], [0.5, 1.0]]), -1),
    (dict(scales=[1.0, 0.0]), -1),
    (dict(dtype=1, n=8, ld=12), -1),        # f16 rows of 24 bytes
    (dict(relax=2.5), -1),                  # relaxed updates only up to 2
    (dict(relax=-0.5), -1),
    (dict(relax=float("nan")), -1),
    (dict(check_inputs=2), -1),             # the new option fields take 0 or 1 ...
    (dict(deterministic=-1), -1),
    (dict(wait_limit_us=-5), -1),           # ... and a non-negative wait bound
    (dict(reserved=1), -1),
    (dict(delta_layout=2), -1),             # unknown Delta layout
    (dict(delta_layout=1, ld=16), -1),      # packed storage needs its own row stride (8 here)
])
def test_invalid_arguments_rejected_before_cuda(call, kw, code):
    assert call.embed(**kw) == code
    assert call.fj.strerror(code)


def test_error_messages_name_the_problem(call):
    assert call.embed(n=5, ld=6) == -1
    assert "16 bytes" in call.fj.strerror(-1)
    assert call.embed(W=[[1.0, 0.5], [0.4, 1.0]]) == -1
    assert "symmetric" in call.fj.strerror(-1)


def test_init_argument_validation(call):
    fj = call.fj
    lib = call.lib
    lib.fjofc_init_cmds.restype = ctypes.c_int

    def init(m=2, n=8, d=2, ld=8, ptr=4096, X=8192, max_iter=0, tol=0.0):
        ptrs = (ctypes.c_void_p * m)(*([ptr] * m))
        opts = fj._InitOpts(max_iter, tol)
        return lib.fjofc_init_cmds(ctypes.c_int32(m), ctypes.c_int64(n), ctypes.c_int32(d), ptrs, ctypes.c_int64(ld),
                                   ctypes.c_int32(0), None, ctypes.c_void_p(X), ctypes.byref(opts), None, None)

    assert init(n=5, ld=6) == -1          # rows not 16-byte aligned
    assert init(X=0) == -1
    assert init(X=8196) == -1             # X not 16-byte aligned
    assert init(d=17) == -6
    assert init(max_iter=-1) == -1
    assert init(tol=-1.0) == -1


def test_oos_argument_validation(call):
    fj = call.fj
    lib = call.lib
    lib.fjofc_oos.restype = ctypes.c_int
    W = np.array([[1.0, 0.5], [0.5, 1.0]])
    opts = fj._Opts(3, -1.0, 1)

    def oos(m=2, n=8, d=2, k=4, ld=8, dptr=4096, X=8192, Y=12288, W=W):
        return lib.fjofc_oos(ctypes.c_int32(m), ctypes.c_int64(n), ctypes.c_int32(d), ctypes.c_int64(k),
                             ctypes.c_void_p(X), ctypes.c_void_p(dptr), ctypes.c_int64(ld), ctypes.c_int32(0), None,
                             np.asarray(W, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             ctypes.c_void_p(Y), None, None, ctypes.byref(opts), None, None)

    assert oos(k=-1) == -1
    assert oos(n=5, ld=6) == -1
    assert oos(dptr=4104) == -1
    assert oos(Y=0) == -1
    assert oos(d=17) == -6
    assert oos(W=[[1.0, 0.5], [0.3, 1.0]]) == -1
    assert oos(k=0) == 0          # nothing to embed: success without touching the GPU

    def oos_form(form, m=2, n=8, d=2):
        o = fj._Opts(3, -1.0, 1)
        o.oos_form = form
        Wm = np.eye(m) + 0.5 * (1 - np.eye(m))
        return lib.fjofc_oos(ctypes.c_int32(m), ctypes.c_int64(n), ctypes.c_int32(d), ctypes.c_int64(4),
                             ctypes.c_void_p(8192), ctypes.c_void_p(4096), ctypes.c_int64(n), ctypes.c_int32(0), None,
                             Wm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(12288), None, None,
                             ctypes.byref(o), None, None)

    assert oos_form(3) == -1                      # unknown form
    assert oos_form(2, d=9) == -6                 # resident form: d <= 8
    assert oos_form(2, n=100000) == -6            # resident form: does not fit in shared memory
    assert "shared memory" in fj.strerror(-6)


def test_packed_size_matches_the_band_layout(call):
    """fjofc_packed_size against the layout written out: bands of 128 rows from the
    diagonal, band b paired with band nB - 1 - b, widths rounded to 16 bytes."""
    lib = call.lib
    lib.fjofc_packed_size.restype = ctypes.c_int64
    lib.fjofc_packed_size.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
    for n, dt, es in [(5000, 0, 4), (5000, 1, 2), (129, 0, 4), (1, 0, 4), (300, 2, 2), (20000, 1, 2)]:
        ld = ctypes.c_int64(0)
        size = lib.fjofc_packed_size(n, dt, ctypes.byref(ld))
        nb = -(-n // 128)
        al = lambda w: -(-w // (16 // es)) * (16 // es)          # noqa: E731
        widths = [al(n - 128 * b) + (al(n - 128 * (nb - 1 - b)) if nb - 1 - b != b else 0)
                  for b in range(0, (nb - 1) // 2 + 1)]
        assert ld.value == max(widths)
        assert size == -(-nb // 2) * 128 * ld.value
        assert size <= n * (n + 256) // 2 + 128 * ld.value       # about half of n^2, one band of slack
    assert lib.fjofc_packed_size(0, 0, None) == -1
    assert lib.fjofc_packed_size(10, 7, None) == -1
