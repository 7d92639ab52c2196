"""Planted mistakes in the oracles, on the CPU: each plausible slip below (a flipped sign,
a dropped term, a wrong index or weight, a transposed operand, the printed form of a
garbled formula) replaces one function of ``oracle.fjofc_oracle`` (or of
``oracle.mlp_oracle``) in a child process, and at least one pin of
``tests/test_oracle_pins.py`` (or ``tests/test_mlp_oracle_pins.py``) must then fail.
This is the evidence that the pins constrain the oracles, not only that the oracles
pass them.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PINS = os.path.join(HERE, "test_oracle_pins.py")
MLP_PINS = os.path.join(HERE, "test_mlp_oracle_pins.py")


def apply(name):
    """Replace one oracle function by its planted-mistake version."""
    from oracle import fjofc_oracle as O
    orig = {k: getattr(O, k) for k in dir(O) if not k.startswith("_")}

    def guttman_B_sign(X, W, Delta):                  # Eq. B with the sign of b_ij flipped
        return -orig["guttman_B"](X, W, Delta)

    def guttman_B_no_diagonal(X, W, Delta):           # Eq. B without its diagonal
        B = orig["guttman_B"](X, W, Delta)
        B[np.diag_indices(B.shape[0])] = 0.0
        return B

    def laplacian_sign(W):                            # L = W - D instead of D - W
        return W - np.diag(W.sum(axis=1))

    def omnibus_unit_commensurability(Wm, n):         # w_ij ignored (taken as 1)
        Wm = np.array(Wm, dtype=np.float64)
        off = ~np.eye(Wm.shape[0], dtype=bool)
        Wm[off] = 1.0
        return orig["omnibus_weights"](Wm, n)

    def stress_ordered_pairs(X, W, Delta):            # sum over i != j instead of i < j
        return 2.0 * orig["raw_stress"](X, W, Delta)

    def modified_weights_m_for_n(Wm, n):              # Eq. modW with m where n belongs
        return orig["modified_weight_matrix"](Wm, np.asarray(Wm).shape[0])

    def stopping_sign(prev, cur, tol, tol_mode, n_pairs):   # the printed sign of the test
        return orig["continue_iterating"](cur, prev, tol, tol_mode, n_pairs)

    def relaxed_away(X, Lp, W, Delta, relax):         # relaxed step in the wrong direction
        G = O.guttman_step(X, Lp, W, Delta)
        return X - relax * (G - X)

    def step_without_pinv(X, Lp, W, Delta):           # L^+ dropped (B X / N)
        return orig["guttman_B"](X, W, Delta) @ X / X.shape[0]

    def cmds_without_centring(D, d):                  # -1/2 D^2 without J ... J
        D = np.asarray(D, dtype=np.float64)
        lam, V = np.linalg.eigh(-0.5 * D * D)
        top = np.argsort(lam)[::-1][:d]
        return V[:, top] * np.sqrt(np.maximum(lam[top], 0.0))

    def procrustes_as_printed(xi, xi0):               # xi U V' (the printed form)
        U, _, Vt = np.linalg.svd(np.asarray(xi0).T @ np.asarray(xi))
        return xi @ (U @ Vt)

    def oos_step_L12_sign(X, delta_new, y, Wm):       # (B12' + L12') X
        mn = X.shape[0]
        Wo, Do, Xo = O.oos_blocks(X, delta_new, y, Wm)
        Lo = O.laplacian(Wo)
        Bo = O.guttman_B(Xo, Wo, Do)
        L22inv = np.linalg.inv(Lo[mn:, mn:])
        return L22inv @ ((Bo[:mn, mn:].T + Lo[:mn, mn:].T) @ X) + L22inv @ (Bo[mn:, mn:] @ y)

    def oos_closed_without_wjj(X, delta_new, y, Wm):  # xi_j, psi_j without w_jj
        Wm = np.asarray(Wm, dtype=np.float64)
        ones = Wm.copy()
        ones[np.diag_indices(Wm.shape[0])] = 1.0
        step = orig["oos_step_closed_form"](X, delta_new, y, ones)
        # keep Wmod^-1 of the true weights, lose only the w_jj factors of xi and psi
        n = np.asarray(X).shape[0] // Wm.shape[0]
        return np.linalg.inv(O.modified_weight_matrix(Wm, n)) @ (O.modified_weight_matrix(ones, n) @ step)

    def oos_stress_without_commensurability(X, delta_new, y, Wm):
        Wm = np.asarray(Wm, dtype=np.float64)
        fid = np.diag(np.diag(Wm))
        return orig["oos_stress_direct"](X, delta_new, y, fid)

    def pinv_default_cutoff(L):                       # numpy's default cutoff
        return np.linalg.pinv(L)

    def guttman_B_unchanged(X, W, Delta):             # the harness's control: no mistake
        return orig["guttman_B"](X, W, Delta)

    from oracle import mlp_oracle as N
    morig = {k: getattr(N, k) for k in dir(N) if not k.startswith("_")}

    def gelu_grad_without_density_term(z):            # Phi(z) only, the z phi(z) term dropped
        return 0.5 * (1.0 + N.erf(z / N.SQRT2))

    def _gradient(theta, X, Y, n_in, hidden, n_out, slip):
        W1, b1, W2, b2, W3, b3 = N.unpack(theta, n_in, hidden, n_out)
        yhat, (X, z1, h1, z2, h2) = N.forward(theta, X, n_in, hidden, n_out)
        B = X.shape[0]
        r = yhat - np.asarray(Y, dtype=np.float64)
        L = float(0.5 * np.sum(r * r) / B)
        dy = r if slip == "no 1/B" else r / B
        gW3 = dy.T @ (h1 if slip == "activation" else h2)
        gb3 = dy.sum(axis=0)
        dz2 = (dy @ W3) * N.gelu_grad(z2)
        gW2 = dz2.T @ h1
        gb2 = dz2.sum(axis=0)
        dz1 = (dz2 @ (W2.T if slip == "transpose" else W2)) * N.gelu_grad(z1)
        gW1 = dz1.T @ X
        gb1 = dz1.sum(axis=0)
        return L, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])

    def gradient_without_batch_mean(theta, X, Y, n_in, hidden, n_out):
        return _gradient(theta, X, Y, n_in, hidden, n_out, "no 1/B")

    def gradient_wrong_activation(theta, X, Y, n_in, hidden, n_out):
        return _gradient(theta, X, Y, n_in, hidden, n_out, "activation")

    def gradient_transposed_weight(theta, X, Y, n_in, hidden, n_out):
        return _gradient(theta, X, Y, n_in, hidden, n_out, "transpose")

    def adam_without_bias_correction(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        return theta - lr * m / (np.sqrt(v) + eps), m, v

    def loss_mean_for_sum(theta, X, Y, n_in, hidden, n_out):   # mean over outputs too
        yhat, _ = N.forward(theta, X, n_in, hidden, n_out)
        r = yhat - np.asarray(Y, dtype=np.float64)
        return float(0.5 * np.mean(r * r))

    def features_one_scale(delta_new, landmarks, inv_mean):    # modality 0's scale for all
        return morig["features"](delta_new, landmarks, np.full(len(inv_mean), inv_mean[0]))

    mlp_table = {
        "GELU' density term dropped": ("gelu_grad", gelu_grad_without_density_term),
        "gradient without 1/B": ("gradient", gradient_without_batch_mean),
        "gradient with the wrong activation": ("gradient", gradient_wrong_activation),
        "gradient with a transposed weight": ("gradient", gradient_transposed_weight),
        "Adam without bias correction": ("adam_step", adam_without_bias_correction),
        "loss as a mean over outputs": ("loss", loss_mean_for_sum),
        "features with one scale": ("features", features_one_scale),
    }
    if name in mlp_table:
        fn_name, fn = mlp_table[name]
        setattr(N, fn_name, fn)
        return sorted(mlp_table)

    table = {
        "B sign": ("guttman_B", guttman_B_sign),
        "B diagonal": ("guttman_B", guttman_B_no_diagonal),
        "Laplacian sign": ("laplacian", laplacian_sign),
        "commensurability weight": ("omnibus_weights", omnibus_unit_commensurability),
        "stress over ordered pairs": ("raw_stress", stress_ordered_pairs),
        "m for n in Wmod": ("modified_weight_matrix", modified_weights_m_for_n),
        "stopping sign": ("continue_iterating", stopping_sign),
        "relaxed direction": ("relaxed_step", relaxed_away),
        "pseudoinverse dropped": ("guttman_step", step_without_pinv),
        "cMDS without double centring": ("cmds", cmds_without_centring),
        "Procrustes as printed": ("procrustes_fit", procrustes_as_printed),
        "out-of-sample L12 sign": ("oos_step", oos_step_L12_sign),
        "out-of-sample w_jj dropped": ("oos_step_closed_form", oos_closed_without_wjj),
        "out-of-sample stress without commensurability": ("oos_stress_direct",
                                                          oos_stress_without_commensurability),
        "pseudoinverse cutoff": ("pseudoinverse", pinv_default_cutoff),
        "control": ("guttman_B", guttman_B_unchanged),
    }
    fn_name, fn = table[name]
    setattr(O, fn_name, fn)
    return sorted(table)


MUTANTS = ["B sign", "B diagonal", "Laplacian sign", "commensurability weight", "stress over ordered pairs",
           "m for n in Wmod", "stopping sign", "relaxed direction", "pseudoinverse dropped",
           "cMDS without double centring", "Procrustes as printed", "out-of-sample L12 sign",
           "out-of-sample w_jj dropped", "out-of-sample stress without commensurability", "pseudoinverse cutoff"]
MLP_MUTANTS = ["GELU' density term dropped", "gradient without 1/B", "gradient with the wrong activation",
               "gradient with a transposed weight", "Adam without bias correction", "loss as a mean over outputs",
               "features with one scale"]


def _run_pins(name, pins=PINS):
    code = (f"import sys; sys.path[:0] = [{ROOT!r}, {HERE!r}]\n"
            "import test_oracle_mutations as M\n"
            f"M.apply({name!r})\n"
            "import pytest\n"
            f"sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', {pins!r}]))\n")
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)


def test_mutant_lists_are_complete():
    from oracle import fjofc_oracle as O
    from oracle import mlp_oracle as N
    saved = [(mod, {k: getattr(mod, k) for k in dir(mod) if not k.startswith("_")}) for mod in (O, N)]
    try:
        assert sorted(MUTANTS + ["control"]) == apply(MUTANTS[0])
        assert sorted(MLP_MUTANTS) == apply(MLP_MUTANTS[0])
    finally:
        for mod, funcs in saved:
            for k, v in funcs.items():
                setattr(mod, k, v)


@pytest.mark.parametrize("name", MUTANTS + MLP_MUTANTS)
def test_planted_mistake_fails_a_pin(name):
    r = _run_pins(name, MLP_PINS if name in MLP_MUTANTS else PINS)
    assert r.returncode == 1, (name, r.returncode, r.stdout[-2000:], r.stderr[-2000:])
    assert "failed" in r.stdout, (name, r.stdout[-2000:])


@pytest.mark.parametrize("pins", [PINS, MLP_PINS])
def test_control_replacement_passes_every_pin(pins):
    """The same harness with a replacement that changes nothing: every pin passes, so a
    failure above comes from the planted mistake."""
    r = _run_pins("control", pins)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-2000:])
