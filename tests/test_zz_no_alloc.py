"""fjofc_embed_noalloc against fjofc_embed, through the C ABI.

fjofc_embed_noalloc serves callers that cannot allocate device memory while they run
(real-time loops that must stay out of every allocator after start-up, processes whose
device memory is partitioned at launch, code that must not fail part-way for lack of
memory).  It runs the same kernels in one fixed device array inside the library.  This
test calls it twice in a row, on two different problems, and checks each result against
fjofc_embed on the same inputs with the parity tolerances (X within relative Frobenius
1e-5, stress within 1e-6 relative); the second call runs in the array the first call
left behind.  It checks that a call after the first one on the device allocates nothing
from the device's stream-ordered memory pool (the allocator fjofc_embed uses), and that
a problem too large for the array is refused.  This file is collected last (its name) so
that a run that stops at the first failure has run every other test first; it also
passes alone.
"""
import ctypes

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import ensure_library
    fj = ensure_library()
    lib = ctypes.CDLL(fj.LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.fjofc_embed_noalloc.argtypes = [i32, i64, i32, ctypes.POINTER(vp), i64, i32, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_double), vp, ctypes.POINTER(fj._Opts),
                                        ctypes.POINTER(fj._Result), vp]
    lib.fjofc_embed_noalloc.restype = ctypes.c_int
    return torch, fj, lib


def _noalloc(torch, fj, lib, deltas, W, X, max_iter, tol, tol_mode):
    m = len(deltas)
    n = int(deltas[0].shape[0])
    d = int(X.shape[1])
    ptrs = (ctypes.c_void_p * m)(*[D.data_ptr() for D in deltas])
    Wn = np.ascontiguousarray(W, dtype=np.float64)
    opts = fj._Opts(max_iter, tol, fj.TOL_RELATIVE if tol_mode == "relative" else fj.TOL_ABS_NORMALIZED, 0)
    hist = np.zeros(max_iter + 1)
    res = fj._Result()
    res.stress_history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.fjofc_embed_noalloc(m, n, d, ptrs, deltas[0].stride(0), fj._dtype_code(deltas[0]), None,
                                 Wn.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(X.data_ptr()),
                                 ctypes.byref(opts), ctypes.byref(res), stream)
    return st, res, hist


def test_noalloc_matches_embed_on_two_consecutive_calls(env):
    torch, fj, lib = env
    problems = [
        dict(k=0, n=300, m=2, d=3, seed=901, iters=25, tol=-1.0),
        dict(k=0, n=517, m=3, d=2, seed=902, iters=400, tol=1e-5),   # stops on the tolerance
    ]
    for spec in problems:
        prob = synthetic.make_insample(spec["k"], n=spec["n"], m=spec["m"], d=spec["d"], seed=spec["seed"])
        dev = [fj.to_device_delta(D) for D in prob.deltas]
        X0 = torch.as_tensor(np.asarray(prob.X0, np.float32)).cuda()

        Xa = X0.clone()
        ref = fj.embed(dev, prob.W, Xa, max_iter=spec["iters"], tol=spec["tol"], tol_mode="relative")
        Xb = X0.clone()
        st, res, hist = _noalloc(torch, fj, lib, dev, prob.W, Xb, spec["iters"], spec["tol"], "relative")
        torch.cuda.synchronize()
        assert st == 0, fj.strerror(st)
        assert res.iters == ref.iters
        a = Xa.double().cpu().numpy()
        b = Xb.double().cpu().numpy()
        assert np.linalg.norm(b - a) / np.linalg.norm(a) <= 1e-5
        assert abs(res.stress - ref.stress) <= 1e-6 * ref.stress
        np.testing.assert_allclose(hist[:res.iters + 1], ref.history, rtol=1e-6)


def test_noalloc_refuses_problems_beyond_its_array(env):
    torch, fj, lib = env
    n = 20000                     # partials alone exceed the fixed array at m = 2, d = 3
    dev = [fj.empty_delta(n) for _ in range(2)]
    X = torch.zeros((2 * n, 3), dtype=torch.float32, device="cuda")
    st, res, _ = _noalloc(torch, fj, lib, dev, synthetic.weights_matrix(2), X, 3, -1.0, "relative")
    assert st == fj.FJOFC_ERR_UNSUPPORTED
    assert "scratch" in fj.strerror(st)


def _cudart():
    import ctypes.util
    for name in (ctypes.util.find_library("cudart"), "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


class _Pool:
    """Used-memory high-water mark of the current device's default memory pool (the pool
    cudaMallocAsync draws from), read and reset through the CUDA runtime."""
    USED_CURRENT, USED_HIGH, RESERVED_CURRENT = 7, 8, 5

    def __init__(self, rt, dev):
        self.rt = rt
        self.pool = ctypes.c_void_p()
        assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(self.pool), ctypes.c_int(dev)) == 0

    def get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolGetAttribute(self.pool, ctypes.c_int(attr), ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolSetAttribute(self.pool, ctypes.c_int(self.USED_HIGH), ctypes.byref(zero)) == 0


def test_noalloc_call_allocates_nothing(env):
    """After the first call on the device (which may load device code), a call leaves the
    pool's used-memory high-water mark where it was; an ordinary fjofc_embed call on the
    same problem raises it (the probe sees the library's allocations)."""
    torch, fj, lib = env
    rt = _cudart()
    if rt is None:
        pytest.skip("CUDA runtime library not found for the memory-pool probe")
    prob = synthetic.make_insample(0, n=700, m=2, d=3, seed=903)
    dev = [fj.to_device_delta(D) for D in prob.deltas]
    X0 = torch.as_tensor(np.asarray(prob.X0, np.float32)).cuda()
    X = X0.clone()
    st, _, _ = _noalloc(torch, fj, lib, dev, prob.W, X, 10, -1.0, "relative")      # start-up call
    assert st == 0, fj.strerror(st)
    torch.cuda.synchronize()
    pool = _Pool(rt, torch.cuda.current_device())
    pool.reset_high()
    used0 = pool.get(_Pool.USED_CURRENT)
    X = X0.clone()
    st, _, _ = _noalloc(torch, fj, lib, dev, prob.W, X, 10, -1.0, "relative")
    torch.cuda.synchronize()
    assert st == 0, fj.strerror(st)
    assert pool.get(_Pool.USED_HIGH) == used0
    assert pool.get(_Pool.USED_CURRENT) == used0
    # control: the allocating entry point draws its scratch from this pool
    X = X0.clone()
    fj.embed(dev, prob.W, X, max_iter=10)
    torch.cuda.synchronize()
    assert pool.get(_Pool.USED_HIGH) > used0
