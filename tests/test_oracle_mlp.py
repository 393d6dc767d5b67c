"""Pins of the surrogate-network oracle (oracle/mlp.py) against definitions that do not
come from the oracle itself: finite differences of the loss, PyTorch's autograd, PyTorch's
BF16 conversion, GELU and Adam, closed forms and brute-force scans."""
import numpy as np
import pytest

from oracle import mlp as M

torch = pytest.importorskip("torch")


def random_problem(n=24, seed=0, scale=0.5):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0.0, scale, M.N_PARAMS)
    x = np.stack([rng.uniform(0.65, 0.95, n), rng.uniform(0, 0.95, n),
                  rng.uniform(0.6, 1.2, n)], axis=1)
    y = np.stack([np.exp(rng.uniform(-6, -2, n)), rng.uniform(5, 9, n),
                  np.exp(rng.uniform(-4, -1, n))], axis=1)
    return theta, x, y, M.normalisation(x, y)


def test_parameter_count_and_layout():
    assert M.N_PARAMS == 3 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3 == 4611
    theta = np.arange(M.N_PARAMS, dtype=float)
    W1, b1, W2, b2, W3, b3 = M.unpack(theta)
    assert W1[1, 0] == 3 and b1[0] == 192 and W2[0, 1] == 257 and b3[-1] == 4610
    assert np.array_equal(M.pack([W1, b1, W2, b2, W3, b3]), theta)


def test_bf16_round_matches_torch_conversion():
    rng = np.random.default_rng(1)
    a = np.concatenate([rng.normal(0, 1, 20000), rng.normal(0, 1e-30, 2000),
                        rng.normal(0, 1e30, 2000)]).astype(np.float32)
    # exact ties of both parities and values one ulp around them
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 2 ** -130 + 2 ** -141],
                    dtype=np.float32)
    a = np.concatenate([a, ties, np.nextafter(ties, np.float32(10)),
                        np.nextafter(ties, np.float32(-10)), np.float32([0, -0.0, 1e-45])])
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    got = M.bf16_round(a)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert M.bf16_round(np.float32(1 + 2 ** -8)) == 1.0            # tie to even (down)
    assert M.bf16_round(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6  # tie to even (up)


def test_gelu_and_its_derivative():
    z = np.linspace(-8, 8, 2001)
    ref = torch.nn.functional.gelu(torch.from_numpy(z), approximate="none").numpy()
    assert np.max(np.abs(M.gelu(z) - ref)) < 1e-14
    assert M.gelu(0.0) == 0.0 and M.gelu(40.0) == 40.0 and abs(M.gelu(-40.0)) < 1e-300
    assert M.gelu_grad(0.0) == pytest.approx(0.5, abs=1e-15)
    h = 1e-5
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(M.gelu_grad(z) - fd)) < 1e-9


def test_gradient_matches_central_differences():
    theta, x, y, norm = random_problem(n=12, seed=2)
    loss, g = M.loss_and_grad(theta, x, y, norm, bf16=False)
    h = 1e-6
    fd = np.empty_like(g)
    for p in range(M.N_PARAMS):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fd[p] = (M.loss_and_grad(tp, x, y, norm, bf16=False)[0]
                 - M.loss_and_grad(tm, x, y, norm, bf16=False)[0]) / (2 * h)
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(g)))
    assert loss > 0


def test_gradient_matches_torch_autograd():
    theta, x, y, norm = random_problem(n=40, seed=3)
    loss, g = M.loss_and_grad(theta, x, y, norm, bf16=False)
    in_m, in_s, out_m, out_s = (torch.tensor(v, dtype=torch.float64) for v in norm)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    sizes = [int(np.prod(s)) for s in M.SIZES]
    W1, b1, W2, b2, W3, b3 = (p.reshape(s) for p, s in zip(th.split(sizes), M.SIZES))
    xt = torch.tensor(x)
    xn = (torch.stack([torch.log(1 - xt[:, 0]), torch.log(1 - xt[:, 1]), xt[:, 2]], dim=1)
          - in_m) / in_s
    a1 = torch.nn.functional.gelu(xn @ W1.T + b1)
    a2 = torch.nn.functional.gelu(a1 @ W2.T + b2)
    o = a2 @ W3.T + b3
    yt = torch.tensor(y)
    t = torch.stack([yt[:, 0].log(), yt[:, 1], yt[:, 2].log()], dim=1)
    lt = (((o - (t - out_m) / out_s)) ** 2).mean()
    lt.backward()
    assert loss == pytest.approx(lt.item(), rel=1e-13)
    assert np.max(np.abs(g - th.grad.numpy())) < 1e-13 * max(1.0, np.max(np.abs(g)))


def test_bf16_forward_uses_rounded_weights():
    theta, x, y, norm = random_problem(n=16, seed=4)
    r = M.bf16_round(theta).astype(np.float64)
    l1, g1 = M.loss_and_grad(theta, x, y, norm, bf16=True)
    l2, g2 = M.loss_and_grad(r, x, y, norm, bf16=False)
    assert l1 == l2 and np.array_equal(g1, g2)
    assert not np.array_equal(r, theta)


def test_forward_closed_form_with_zero_hidden_weights():
    theta, x, y, norm = random_problem(n=5, seed=5)
    W1, b1, W2, b2, W3, b3 = M.unpack(theta)
    b3 = np.array([0.25, -0.5, 1.0])
    W3 = np.zeros_like(W3)
    t = M.pack([W1, b1, W2, b2, W3, b3])
    pred, o, _ = M.forward(t, x, norm, bf16=False)
    out_m, out_s = norm[2], norm[3]
    expect = b3 * out_s + out_m
    assert np.allclose(o, b3)
    assert np.allclose(pred[:, 0], np.exp(expect[0]))
    assert np.allclose(pred[:, 1], expect[1])
    assert np.allclose(pred[:, 2], np.exp(expect[2]))


def test_normalisation_standardises_the_data():
    theta, x, y, norm = random_problem(n=50, seed=6)
    in_m, in_s, out_m, out_s = norm
    xn = (M.features(x) - in_m) / in_s
    assert np.allclose(xn.mean(0), 0, atol=1e-13) and np.allclose(xn.std(0), 1)
    t = (M.to_net_targets(y) - out_m) / out_s
    assert np.allclose(t.mean(0), 0, atol=1e-13) and np.allclose(t.std(0), 1)
    x[:, 2] = 0.8
    assert M.normalisation(x, y)[1][2] == 1.0
    assert np.allclose(M.from_net_outputs(M.to_net_targets(y)), y)


def test_adam_matches_torch_optimizer():
    rng = np.random.default_rng(7)
    p0 = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(6)]
    tp = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    th, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for k, g in enumerate(grads, start=1):
        th, m, v = M.adam_step(th, m, v, g, k, 3e-3)
        tp.grad = torch.tensor(g)
        opt.step()
    assert np.max(np.abs(th - tp.detach().numpy())) < 1e-15
    # the first step moves every parameter by lr against the sign of its gradient
    th1, _, _ = M.adam_step(p0, np.zeros(50), np.zeros(50), grads[0], 1, 1e-3)
    assert np.allclose(p0 - th1, 1e-3 * np.sign(grads[0]), rtol=1e-6)


def test_inversion_finds_the_crossing_a_scan_brackets():
    theta, x, y, norm = random_problem(n=64, seed=8, scale=0.1)
    # make theta strictly decreasing in kappa: only the ln(1 - kappa) feature reaches the
    # hidden layers, with positive weights, through units kept on GELU's increasing branch
    # (z > 0 there) and positive output weights
    W1, b1, W2, b2, W3, b3 = M.unpack(theta)
    W1[:, 0] = 0.0
    W1[:, 2] = 0.0
    W1[:, 1] = np.abs(W1[:, 1]) * 0.1 + 0.01
    b1[:] = 1.0
    W2 = np.abs(W2)
    b2[:] = 0.0
    W3[0] = np.abs(W3[0]) + 0.01
    t = M.pack([W1, b1, W2, b2, W3, b3])
    ks = np.linspace(0, 0.95, 951)
    q = np.stack([np.full_like(ks, 0.8), ks, np.full_like(ks, 0.9)], axis=1)
    th = M.forward(t, q, norm)[0][:, 0]
    assert np.all(np.diff(th) < 0)
    assert np.isnan(M.invert_kappa(t, norm, 0.8, 0.9, th[0] * 1.01))
    assert np.isnan(M.invert_kappa(t, norm, 0.8, 0.9, th[-1] * 0.99))
    for target in (th[100] * 0.999, th[500], th[900] * 1.001):
        k = M.invert_kappa(t, norm, 0.8, 0.9, target)
        i = np.searchsorted(-th, -target)          # first grid point with theta <= target
        assert ks[i - 1] <= k <= ks[i] + 1e-9


def test_features_closed_form():
    x = np.array([[0.0, 0.0, 0.7], [0.5, 0.75, 1.1], [1 - np.exp(-3), 1 - np.exp(-2), 0.6]])
    f = M.features(x)
    assert np.allclose(f, [[0, 0, 0.7], [np.log(0.5), np.log(0.25), 1.1], [-3, -2, 0.6]],
                       atol=1e-15)
