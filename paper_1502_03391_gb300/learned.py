"""Learned warm start for out-of-sample embedding (argument marshalling only).

The paper has no learned component; this is the learned form added beside the method.
A network with two hidden GELU layers maps a new object's dissimilarities to fixed
in-sample landmarks (float16 inputs, one normaliser per modality) to a start for the
out-of-sample Guttman iterations of Sec. 3 (``fjofc_oos``), which refine it.  Two output
heads are supported: n_out = m*d predicts every modality's position y_j (the default:
on the synthetic workloads the modalities' solutions lie far apart, so one shared
position is no better than the standard start), n_out = d predicts the commensurate
position ybar = mean_j y_j, used for every modality.  Per object the start with the
lower out-of-sample stress is kept, so the warm start never starts worse than the
standard one.  Training targets are the method's own out-of-sample solutions.  Every
step (features, forward, backward, Adam, the broadcast and the choice of start) runs
in the library's kernels.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional, Sequence

import numpy as np

from . import _lib, _check, _stream_handle, _torch, oos as _oos

_vp, _i32, _i64, _u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64


class TrainOpts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("reserved", ctypes.c_int32 * 4)]


_lib.fjofc_mlp_param_count.argtypes = [_i32, _i32, _i32]
_lib.fjofc_mlp_param_count.restype = _i64
_lib.fjofc_mlp_init.argtypes = [_vp, _i32, _i32, _i32, _u64, _vp]
_lib.fjofc_mlp_features.argtypes = [_i32, _i64, _i64, _vp, _i64, _vp, _i32, ctypes.POINTER(ctypes.c_float), _vp, _vp]
_lib.fjofc_mlp_forward.argtypes = [_vp, _i32, _i32, _i32, _vp, _i64, _vp, _vp]
_lib.fjofc_mlp_gradient.argtypes = [_vp, _i32, _i32, _i32, _vp, _vp, _i64, _vp, ctypes.POINTER(ctypes.c_double), _vp]
_lib.fjofc_mlp_train.argtypes = [_vp, _i32, _i32, _i32, _vp, _vp, _i64, ctypes.POINTER(TrainOpts),
                                 ctypes.POINTER(ctypes.c_float), _vp]
_lib.fjofc_mlp_broadcast.argtypes = [_i64, _i32, _i32, _vp, _vp, _vp]
_lib.fjofc_mlp_select.argtypes = [_i64, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp]
for _f in ("fjofc_mlp_init", "fjofc_mlp_features", "fjofc_mlp_forward", "fjofc_mlp_gradient", "fjofc_mlp_train",
           "fjofc_mlp_broadcast", "fjofc_mlp_select"):
    getattr(_lib, _f).restype = ctypes.c_int


def _ptr(t):
    return _vp(t.data_ptr()) if t is not None else None


def choose_landmarks(n: int, count: int = 256, seed: int = 0) -> np.ndarray:
    """``count`` distinct in-sample indices drawn uniformly with a seeded generator."""
    return np.sort(np.random.default_rng([int(seed), 4211]).choice(n, size=min(count, n), replace=False)).astype(
        np.int32)


def features(delta_new, landmarks, inv_mean: Sequence[float], stream=None):
    """float16 (k, m*L) network inputs from a (k, m, n) out-of-sample dissimilarity view."""
    torch = _torch()
    k, m, n = (int(s) for s in delta_new.shape)
    lm = torch.as_tensor(np.asarray(landmarks, np.int32), device=delta_new.device)
    out = torch.empty((k, m * lm.numel()), dtype=torch.float16, device=delta_new.device)
    im = (ctypes.c_float * m)(*[float(v) for v in inv_mean])
    _check(_lib.fjofc_mlp_features(m, n, k, _ptr(delta_new), delta_new.stride(1), _ptr(lm), lm.numel(), im,
                                   _ptr(out), _stream_handle(stream, delta_new.device)))
    return out


@dataclasses.dataclass
class WarmStartResult:
    Y: object               # (k, m, d) chosen starts
    used_warm: object       # int32 (k,) 1 where the network's start was kept
    stress_warm: object     # float64 (k,) stress of the network's start
    stress_std: object      # float64 (k,) stress of the standard start


class WarmStartMLP:
    """Parameters of the network on one CUDA device and the calls that use them."""

    def __init__(self, n_in: int, hidden: int, n_out: int, seed: int = 0, device="cuda", stream=None):
        torch = _torch()
        self.dims = (int(n_in), int(hidden), int(n_out))
        P = _lib.fjofc_mlp_param_count(*self.dims)
        if P < 0:
            raise ValueError("invalid network sizes")
        self.params = torch.empty(int(P), dtype=torch.float32, device=device)
        _check(_lib.fjofc_mlp_init(_ptr(self.params), *self.dims, int(seed), _stream_handle(stream, self.params.device)))

    def forward(self, x, stream=None):
        torch = _torch()
        out = torch.empty((int(x.shape[0]), self.dims[2]), dtype=torch.float32, device=x.device)
        _check(_lib.fjofc_mlp_forward(_ptr(self.params), *self.dims, _ptr(x), int(x.shape[0]), _ptr(out),
                                      _stream_handle(stream, x.device)))
        return out

    def gradient(self, x, y, stream=None):
        torch = _torch()
        g = torch.empty_like(self.params)
        loss = ctypes.c_double(0.0)
        _check(_lib.fjofc_mlp_gradient(_ptr(self.params), *self.dims, _ptr(x), _ptr(y), int(x.shape[0]), _ptr(g),
                                       ctypes.byref(loss), _stream_handle(stream, x.device)))
        return loss.value, g

    def train(self, x, y, epochs: int, batch: int = 256, lr: float = 1e-3, seed: int = 0, stream=None) -> np.ndarray:
        opts = TrainOpts(int(epochs), int(batch), float(lr), 0.9, 0.999, 1e-8, int(seed))
        hist = (ctypes.c_float * max(int(epochs), 1))()
        _check(_lib.fjofc_mlp_train(_ptr(self.params), *self.dims, _ptr(x), _ptr(y), int(x.shape[0]),
                                    ctypes.byref(opts), hist, _stream_handle(stream, x.device)))
        return np.array(hist[:int(epochs)], dtype=np.float64)

    def warm_start(self, X, delta_new, weights, Y_std, landmarks, inv_mean, stream=None) -> WarmStartResult:
        """Starts for fjofc_oos: the network's start where its out-of-sample stress is not
        above the standard start's, else the standard start (``Y_std``, (k, m, d), left
        unchanged)."""
        torch = _torch()
        k, m, d = (int(s) for s in Y_std.shape)
        x = features(delta_new, landmarks, inv_mean, stream)
        yhat = self.forward(x, stream)
        h = _stream_handle(stream, Y_std.device)
        if self.dims[2] == m * d:                   # one position per modality
            Yw = yhat.view(k, m, d)
        elif self.dims[2] == d:                     # one shared position
            Yw = torch.empty_like(Y_std)
            _check(_lib.fjofc_mlp_broadcast(k, m, d, _ptr(yhat), _ptr(Yw), h))
        else:
            raise ValueError("the network's output must have d or m*d values")
        sw = torch.empty(k, dtype=torch.float64, device=Y_std.device)
        ss = torch.empty(k, dtype=torch.float64, device=Y_std.device)
        Ytmp = Yw.clone()
        _oos(X, delta_new, weights, Ytmp, max_iter=0, stress_out=sw, stream=stream)
        Ytmp.copy_(Y_std)
        _oos(X, delta_new, weights, Ytmp, max_iter=0, stress_out=ss, stream=stream)
        used = torch.empty(k, dtype=torch.int32, device=Y_std.device)
        Y = Y_std.clone()
        _check(_lib.fjofc_mlp_select(k, m, d, _ptr(Yw), _ptr(sw), _ptr(ss), _ptr(Y), _ptr(used), h))
        return WarmStartResult(Y, used, sw, ss)
