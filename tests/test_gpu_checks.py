"""GPU tests of the in-sample loop's input check (fjofc_opts.check_inputs) and of its
bounded-wait error path (fjofc_opts.wait_limit_us), through the C ABI.

* check_inputs: Delta must hold dissimilarities (Sec. 1.2: finite, non-negative,
  symmetric).  A valid input gives bitwise the same result as an unchecked call; an
  asymmetric, negative or non-finite entry returns FJOFC_ERR_ARG naming the first bad
  entry in (modality, row, column) order, and X is left as given.
* Bounded waits: a test hook makes the first grid-wide wait of the next loop expect one
  arrival more than its CTAs make.  No kernel faults or hangs: every CTA gives up after
  the 1 ms bound, waits for its own copies in flight and returns; the call reports
  FJOFC_ERR_TIMEOUT at the phase-C wait (site 32) with X as given, and the next
  ordinary call on the same device matches the oracle.
"""
import numpy as np
import pytest

from oracle import fjofc_oracle as O
import synthetic
from parity_rule import X_TOL, assert_history, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fj():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import ensure_library
    return ensure_library()


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _embed(fj, deltas, W, X0, iters, **kw):
    import torch
    dev = [fj.to_device_delta(D) for D in deltas]
    X = torch.as_tensor(np.asarray(X0, np.float32)).cuda().contiguous()
    res = fj.embed(dev, W, X, max_iter=iters, check=False, **kw)
    torch.cuda.synchronize()
    return X.cpu().numpy(), res


def test_check_inputs_passes_valid_input_unchanged(fj):
    prob = synthetic.make_insample(0, n=333, m=3, d=3, seed=1301)
    Xa, ra = _embed(fj, prob.deltas, prob.W, prob.X0, 12)
    Xb, rb = _embed(fj, prob.deltas, prob.W, prob.X0, 12, check_inputs=True)
    assert ra.status == 0 and rb.status == 0
    np.testing.assert_array_equal(Xa, Xb)
    np.testing.assert_array_equal(ra.history, rb.history)
    assert rb.launches == ra.launches + 1


@pytest.mark.parametrize("kind", ["asymmetric", "negative", "nan", "inf"])
def test_check_inputs_rejects_non_dissimilarities(fj, kind):
    n, m = 150, 2
    prob = synthetic.make_insample(0, n=n, m=m, d=2, seed=1302)
    deltas = [D.copy() for D in prob.deltas]
    # two bad entries; the one first in (modality, row, column) order is reported
    if kind == "asymmetric":
        deltas[1][40][90] += 1e-3            # upper entry only
        deltas[1][100][120] += 1.0
        want = ("Delta_2[40][90]", "differs")
    elif kind == "negative":
        deltas[0][70][5] = -1.0              # lower-triangle entry
        deltas[0][5][70] = -1.0
        deltas[1][1][2] = -3.0
        want = ("Delta_1[5][70]", "negative")
    else:
        bad = np.nan if kind == "nan" else np.inf
        deltas[1][149][148] = bad            # last row, below the diagonal
        want = ("Delta_2[149][148]", "not finite")
    X0 = _f32(prob.X0)
    X, res = _embed(fj, deltas, prob.W, X0, 10, check_inputs=True)
    assert res.status == fj.FJOFC_ERR_ARG
    msg = fj.strerror(fj.FJOFC_ERR_ARG)
    assert want[0] in msg and want[1] in msg, msg
    np.testing.assert_array_equal(X, np.asarray(X0, np.float32))
    # the diagonal is not checked (its weight is zero, Eq. W)
    clean = [D.copy() for D in prob.deltas]
    np.fill_diagonal(clean[0], -5.0)
    _, ok = _embed(fj, clean, prob.W, X0, 2, check_inputs=True)
    assert ok.status == 0


def test_wait_limit_error_path_and_recovery(fj):
    prob = synthetic.make_insample(0, n=1500, m=2, d=3, seed=1303)
    X0 = _f32(prob.X0)
    fj.test_barrier_skew(1)
    X, res = _embed(fj, prob.deltas, prob.W, X0, 20, wait_limit_us=1000)
    assert res.status == fj.FJOFC_ERR_TIMEOUT, res.status
    assert "site 32" in fj.strerror(fj.FJOFC_ERR_TIMEOUT)
    np.testing.assert_array_equal(X, np.asarray(X0, np.float32))
    # the hook was consumed: the next call on the same device runs normally
    X, res = _embed(fj, prob.deltas, prob.W, X0, 20)
    assert res.status == 0 and res.iters == 20
    d32 = [_f32(D) for D in prob.deltas]
    ref = O.jofc_embed(d32, prob.W, X0, max_iter=20, keep_iterates=True)
    assert rel_fro(X, ref.X) <= X_TOL
    assert_history(res.history, ref.stress, d32, prob.W, ref.iterates)
