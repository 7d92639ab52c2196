"""GPU tests of the learned warm start (paper_1502_03391_gb300.learned) against the float64
network oracle (oracle/mlp_oracle.py), through the C ABI.

* features: bit-exact against the oracle's formula evaluated in float32 and rounded to
  float16 (the same precision decides the rounding on both sides);
* forward (relative 1e-5) and gradient (relative 1e-4, float32 arithmetic against
  float64) of the full-size 512-512-512-5 network, plus a directional central
  difference of the device loss;
* one Adam step against the oracle's;
* training lowers the loss;
* gain: on a reduced in-sample problem, the trained network's starts (m*d head) need
  fewer out-of-sample iterations to the relative tolerance than the standard start,
  reach the same final stress within 1e-3, and never start above the standard start's
  stress.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fj():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import ensure_library
    return ensure_library()


@pytest.fixture(scope="module")
def L(fj):
    from paper_1502_03391_gb300 import learned
    return learned


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _half_inputs(rng, B, n_in):
    import torch
    x = torch.as_tensor(rng.normal(scale=1.0, size=(B, n_in)).astype(np.float16)).cuda()
    return x, x.double().cpu().numpy()


def test_features_bit_exact(fj, L):
    import torch
    rng = np.random.default_rng(5)
    k, m, n = 37, 2, 301
    dnew = fj.empty_oos_delta(k, m, n)
    host = rng.uniform(0.0, 40.0, size=(k, m, n)).astype(np.float32)
    dnew.copy_(torch.as_tensor(host))
    lm = L.choose_landmarks(n, 64, seed=3)
    inv_mean = [np.float32(1 / 17.3), np.float32(1 / 9.1)]
    got = L.features(dnew, lm, inv_mean).cpu().numpy()
    want = np.empty((k, m * len(lm)), dtype=np.float16)
    for j in range(m):
        want[:, j * len(lm):(j + 1) * len(lm)] = (host[:, j, :][:, lm] * np.float32(inv_mean[j])).astype(np.float16)
    assert got.dtype == np.float16
    np.testing.assert_array_equal(got.view(np.uint16), want.view(np.uint16))
    # and the float64 definition up to the float16 rounding
    ref = M.features(host.astype(np.float64), lm, np.asarray(inv_mean, np.float64))
    np.testing.assert_allclose(got.astype(np.float64), ref, rtol=2 ** -10)


@pytest.mark.parametrize("dims", [(512, 512, 5), (40, 72, 3)])
def test_forward_and_gradient_match_oracle(fj, L, dims):
    import torch
    rng = np.random.default_rng(11)
    net = L.WarmStartMLP(*dims, seed=9)
    theta = net.params.double().cpu().numpy()
    B = 64
    x, xh = _half_inputs(rng, B, dims[0])
    y = rng.normal(size=(B, dims[2])).astype(np.float32)
    yt = torch.as_tensor(y).cuda()
    want_y, _ = M.forward(theta, xh, *dims)
    got_y = net.forward(x).double().cpu().numpy()
    assert _rel(got_y, want_y) <= 1e-5
    loss, g = net.gradient(x, yt)
    want_loss, want_g = M.gradient(theta, xh, y.astype(np.float64), *dims)
    assert abs(loss - want_loss) <= 1e-5 * want_loss
    g = g.double().cpu().numpy()
    assert _rel(g, want_g) <= 1e-4
    # per block (a dropped or mis-indexed block would hide in the global norm)
    offs = np.cumsum([0, dims[1] * dims[0], dims[1], dims[1] * dims[1], dims[1], dims[2] * dims[1], dims[2]])
    for a, b in zip(offs[:-1], offs[1:]):
        assert _rel(g[a:b], want_g[a:b]) <= 1e-4


def test_gradient_directional_difference(fj, L):
    import torch
    rng = np.random.default_rng(12)
    dims = (64, 96, 4)
    net = L.WarmStartMLP(*dims, seed=2)
    x, _ = _half_inputs(rng, 32, dims[0])
    y = torch.as_tensor(rng.normal(size=(32, dims[2])).astype(np.float32)).cuda()
    _, g = net.gradient(x, y)
    u = torch.as_tensor(rng.normal(size=net.params.numel()).astype(np.float32)).cuda()
    u /= u.norm()
    h = 1e-2
    base = net.params.clone()
    net.params.copy_(base + h * u)
    lp, _ = net.gradient(x, y)
    net.params.copy_(base - h * u)
    lm, _ = net.gradient(x, y)
    net.params.copy_(base)
    fd = (lp - lm) / (2 * h)
    dd = float((g * u).sum().item())
    assert abs(fd - dd) <= 2e-2 * abs(dd) + 1e-6


def test_one_adam_step_matches_oracle(fj, L):
    import torch
    rng = np.random.default_rng(13)
    dims = (48, 64, 5)
    net = L.WarmStartMLP(*dims, seed=4)
    theta0 = net.params.double().cpu().numpy()
    B = 128
    x, xh = _half_inputs(rng, B, dims[0])
    y = rng.normal(size=(B, dims[2])).astype(np.float32)
    _, g = M.gradient(theta0, xh, y.astype(np.float64), *dims)
    lr = 1e-3
    # one epoch of one full batch (the epoch order only permutes the rows of the batch)
    net.train(x, torch.as_tensor(y).cuda(), epochs=1, batch=B, lr=lr, seed=1)
    want, _, _ = M.adam_step(theta0, g, np.zeros_like(g), np.zeros_like(g), 1, lr)
    got = net.params.double().cpu().numpy()
    # the first step is lr * g / (|g| + eps): equal up to the float32 gradient's error
    np.testing.assert_allclose(got - theta0, want - theta0, atol=lr * 2e-3)


def test_training_lowers_the_loss(fj, L):
    import torch
    rng = np.random.default_rng(14)
    dims = (64, 128, 3)
    N = 4096
    x, xh = _half_inputs(rng, N, dims[0])
    A = rng.normal(size=(dims[0], dims[2])) / 8.0
    y = torch.as_tensor(np.tanh(xh @ A).astype(np.float32)).cuda()
    net = L.WarmStartMLP(*dims, seed=7)
    l0, _ = net.gradient(x[:1024], y[:1024])
    hist = net.train(x, y, epochs=25, batch=256, lr=2e-3, seed=5)
    l1, _ = net.gradient(x[:1024], y[:1024])
    assert np.all(np.isfinite(hist))
    assert l1 < 0.2 * l0, (l0, l1, hist)


def test_warm_start_gain(fj, L):
    """Reduced version of the learned out-of-sample workload: m=2, n=2000, d=5."""
    import torch
    prob = synthetic.make_insample(4, n=2000)
    m, n, d = prob.spec.m, prob.spec.n, prob.spec.d
    dev = [fj.to_device_delta(D) for D in prob.deltas]
    X = torch.as_tensor(np.asarray(prob.X0, np.float32)).cuda()
    fj.embed(dev, prob.W, X, max_iter=200, tol=1e-7)
    inv_mean = [1.0 / float(D[np.triu_indices(n, 1)].mean()) for D in prob.deltas]
    lm = L.choose_landmarks(n, 256, seed=1)

    def objects(count, stream):
        F_new, dn, Y0 = synthetic.make_oos_objects(prob, count, stream=stream)
        dnew = fj.empty_oos_delta(count, m, n)
        dnew.copy_(torch.as_tensor(dn.astype(np.float32)))
        return dnew, torch.as_tensor(np.asarray(Y0, np.float32)).cuda().contiguous()

    def solve(dnew, Y):
        it = torch.zeros(Y.shape[0], dtype=torch.int32, device="cuda")
        st = torch.zeros(Y.shape[0], dtype=torch.float64, device="cuda")
        fj.oos(X, dnew, prob.W, Y, max_iter=500, tol=1e-6, iters_out=it, stress_out=st)
        return it.cpu().numpy(), st.cpu().numpy()

    # training targets: the method's own solutions from the standard start (every
    # modality's position: the m*d head)
    dtr, Ytr = objects(4000, 1)
    solve(dtr, Ytr)
    target = Ytr.reshape(Ytr.shape[0], m * d).contiguous()
    net = L.WarmStartMLP(m * len(lm), 512, m * d, seed=3)
    hist = net.train(L.features(dtr, lm, inv_mean), target, epochs=40, batch=256, lr=1e-3, seed=2)
    assert hist[-1] < 0.25 * hist[0]

    dte, Y0 = objects(2000, 2)
    ws = net.warm_start(X, dte, prob.W, Y0, lm, inv_mean)
    assert bool((ws.stress_warm.where(ws.used_warm.bool(), ws.stress_std) <= ws.stress_std).all())
    it_std, s_std = solve(dte, Y0.clone())
    it_warm, s_warm = solve(dte, ws.Y)
    used = ws.used_warm.cpu().numpy()
    print(f"warm start kept for {used.mean():.3f} of objects; mean iterations {it_warm.mean():.1f} vs "
          f"{it_std.mean():.1f}; mean final stress {s_warm.mean():.6e} vs {s_std.mean():.6e}")
    assert it_warm.mean() < 0.8 * it_std.mean()
    assert s_warm.mean() <= s_std.mean() * (1 + 1e-3)
