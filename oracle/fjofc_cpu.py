"""ctypes wrapper of ``fjofc_cpu.c``: Algorithm 2 (fJOFC) in float64 on the host cores.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the CPU baseline that
``bench.py`` times beside the GPU path, checked against the numpy oracle by
``tests/test_cpu_fjofc.py``.  ``build()`` compiles the C file with gcc (OpenMP when the
compiler has it) into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fjofc_cpu.c")
OUT = os.path.join(HERE, "_build", "libfjofc_cpu.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the CPU fJOFC library (skipped when it is newer than its source)."""
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    base = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", OUT + ".tmp", SRC, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:                      # no OpenMP: the same code, serial
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"gcc failed for {SRC}:\n{r.stderr}")
    os.replace(OUT + ".tmp", OUT)
    return OUT


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(OUT)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.fjofc_cpu_embed.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_int, ctypes.POINTER(dp), dp, dp,
                                        ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int)]
        lib.fjofc_cpu_embed.restype = ctypes.c_int
        lib.fjofc_cpu_threads.argtypes = []
        lib.fjofc_cpu_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    """Host threads the library's parallel loops use."""
    return int(_load().fjofc_cpu_threads())


def cpu_embed(deltas: Sequence[np.ndarray], Wm: np.ndarray, X0: np.ndarray, max_iter: int, tol: float = -1.0,
              tol_mode: str = "relative"):
    """Algorithm 2's loop from ``X0`` in float64: returns (X, iters, stress history)."""
    lib = _load()
    m = len(deltas)
    n = int(np.asarray(deltas[0]).shape[0])
    D = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in deltas]
    dp = ctypes.POINTER(ctypes.c_double)
    ptrs = (dp * m)(*[x.ctypes.data_as(dp) for x in D])
    W = np.ascontiguousarray(np.asarray(Wm, dtype=np.float64))
    X = np.array(X0, dtype=np.float64, order="C", copy=True)
    d = X.shape[1]
    hist = np.zeros(max_iter + 1)
    it = ctypes.c_int(0)
    rc = lib.fjofc_cpu_embed(m, n, d, ptrs, W.ctypes.data_as(dp), X.ctypes.data_as(dp), int(max_iter), float(tol),
                             1 if tol_mode == "relative" else 0, hist.ctypes.data_as(dp), ctypes.byref(it))
    if rc != 0:
        raise ValueError(f"fjofc_cpu_embed failed ({rc})")
    return X, int(it.value), hist[:it.value + 1]
