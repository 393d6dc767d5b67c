"""The surrogate network's CUDA kernels (lb_mlp_*) against the FP64 oracle (oracle/mlp.py):
normalisation, loss and gradient, Adam steps, inference and the kappa inversion, on
seeded random parameters and data; determinism of graph-replayed training; argument
errors. Both sides use the same BF16-rounded weights (the oracle rounds the same FP32
master values), so the differences left are FP32 accumulation, the FP32 copy of the
normalisation and FP32 erf / exp: tolerances below are 100x the expected size of those."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_1306_6445_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_6445_gb300 import _build

    _build.build()
    from paper_1306_6445_gb300 import lbm as mod

    mod.load_library()
    return mod


def net_with(lbm, n, seed, max_samples=None):
    x, y = I.mlp_random_data(n, seed)
    theta = I.mlp_init(seed + 1)
    net = lbm.MLP(max_samples or n)
    net.set_params(theta)
    net.set_data(x, y)
    return net, theta, x.astype(np.float64), y.astype(np.float64)


# 1: one sample; 17: a ragged tile; 512: 32 CTAs; 6000: more tiles than CTAs (304 x 16)
@pytest.mark.parametrize("n", [1, 17, 512, 6000])
def test_normalisation_loss_and_gradient_match_oracle(lbm, n):
    net, theta, x, y = net_with(lbm, n, seed=10 + n)
    norm = M.normalisation(x, y)
    got = net.norm()
    for a, b in zip(got, norm):
        assert np.allclose(a, b, rtol=1e-6, atol=1e-7)
    loss, g = net.loss_grad()
    lref, gref = M.loss_and_grad(theta.astype(np.float64), x, y, norm, bf16=True)
    assert loss == pytest.approx(lref, rel=1e-4)
    scale = np.max(np.abs(gref))
    assert np.max(np.abs(g - gref)) <= 1e-4 * scale
    # every block of the layout is exercised (no block silently zero)
    k = 0
    for s in M.SIZES:
        sz = int(np.prod(s))
        if n > 1:
            assert np.any(g[k:k + sz] != 0)
        k += sz
    net.close()


def test_gradient_is_deterministic(lbm):
    net, *_ = net_with(lbm, 3000, seed=3)
    a = net.loss_grad()[1]
    b = net.loss_grad()[1]
    assert np.array_equal(a, b)
    net.close()


def test_adam_steps_match_oracle(lbm):
    n, lr, k = 700, 1e-3, 4
    net, theta, x, y = net_with(lbm, n, seed=21)
    norm = M.normalisation(x, y)
    th = theta.astype(np.float64)
    m, v = np.zeros_like(th), np.zeros_like(th)
    losses = []
    for step in range(1, k + 1):
        # the oracle updates an FP32 master copy too: round after each step
        l, g = M.loss_and_grad(th, x, y, norm, bf16=True)
        losses.append(l)
        th, m, v = M.adam_step(th, m, v, g, step, lr)
        th = th.astype(np.float32).astype(np.float64)
    last = net.train(k, lr)
    got = net.params().astype(np.float64)
    assert last == pytest.approx(losses[-1], rel=1e-4)
    d = np.abs((got - theta) - (th - theta))
    # a gradient entry near zero can take either sign on the two sides; Adam then moves
    # it by up to lr in opposite directions. Nearly all entries agree far more closely.
    assert np.mean(d <= 1e-2 * lr) >= 0.99
    assert np.max(d) <= 2 * k * lr
    assert net.steps_done == k
    net.close()


def test_graph_replay_equals_single_steps(lbm):
    a, *_ = net_with(lbm, 900, seed=5)
    b, *_ = net_with(lbm, 900, seed=5)
    la = a.train(50 + 7, 2e-3)                 # one graph replay plus direct launches
    for _ in range(57):
        lb_ = b.train(1, 2e-3)
    assert np.array_equal(a.params(), b.params()) and la == lb_
    a.close()
    b.close()


def test_training_fits_a_smooth_map(lbm):
    """Full-batch Adam on a smooth synthetic map of the sweep's shape (sigma falling
    linearly in kappa and as (1 - T)^1.5, rho_l and rho_v smooth in T) reaches < 1 %."""
    rng = np.random.default_rng(7)
    n = 1024
    x = np.stack([rng.uniform(0.65, 0.95, n), rng.uniform(0, 0.95, n), rng.uniform(0.6, 1.2, n)],
                 axis=1)

    def f(x):
        t, k, tau = x.T
        return np.stack([0.06 * (1 - k) * (1 - t) ** 1.5 * (1 + 0.02 * (tau - 0.9)),
                         0.55 - 0.8 * (t - 0.65) ** 2, 0.002 + 0.3 * (t - 0.6) ** 2], axis=1)

    net = lbm.MLP(n)
    net.set_params(I.mlp_init(3))
    net.set_data(x, f(x))
    l0 = net.loss_grad()[0]
    for steps, lr in ((3000, 3e-3), (3000, 1e-3), (3000, 3e-4)):
        loss = net.train(steps, lr)
    assert loss < 1e-3 * l0
    xt = np.stack([rng.uniform(0.67, 0.93, 256), rng.uniform(0.02, 0.93, 256),
                   rng.uniform(0.62, 1.18, 256)], axis=1)
    err = np.abs(net.forward(xt) / f(xt) - 1)
    assert np.max(err) < 0.02 and np.median(err) < 0.005
    net.close()


def test_forward_matches_oracle(lbm):
    net, theta, x, y = net_with(lbm, 300, seed=31)
    norm = M.normalisation(x, y)
    q = I.mlp_random_data(4097, seed=32)[0]        # ragged final block
    got = net.forward(q)
    ref = M.forward(theta.astype(np.float64), q.astype(np.float64), norm)[0]
    assert np.max(np.abs(got / ref - 1)) < 2e-4
    assert net.forward(np.zeros((0, 3))).shape == (0, 3)
    net.close()


def monotone_params(seed):
    """Random parameters made so that sigma strictly decreases with kappa: only the
    ln(1 - kappa) feature reaches the hidden layers, with positive weights, through units on
    GELU's increasing branch (z > 0), and the sigma output weights are positive."""
    theta = I.mlp_init(seed).astype(np.float64)
    W1, b1, W2, b2, W3, b3 = M.unpack(theta)
    W1[:, 0] = 0.0
    W1[:, 2] = 0.0
    W1[:, 1] = np.abs(W1[:, 1]) * 0.1 + 0.01
    b1[:] = 1.0
    W2 = np.abs(W2) * 0.1          # keeps sigma within about [0.8, 3.8] over kappa
    b2[:] = 0.0
    W3[0] = np.abs(W3[0]) + 0.01
    return M.pack([W1, b1, W2, b2, W3, b3]).astype(np.float32)


def test_invert_kappa_matches_oracle(lbm):
    x, y = I.mlp_random_data(200, seed=41)
    theta = monotone_params(42)
    net = lbm.MLP(200)
    net.set_params(theta)
    net.set_data(x, y)
    norm = M.normalisation(x.astype(np.float64), y.astype(np.float64))
    th64 = theta.astype(np.float64)
    hi_lo = M.forward(th64, np.array([[0.8, 0.0, 0.9], [0.8, 0.95, 0.9]]), norm)[0][:, 0]
    targets = np.exp(np.linspace(np.log(hi_lo[1]) + 0.01, np.log(hi_lo[0]) - 0.01, 9))
    q = np.stack([np.full(9, 0.8), np.full(9, 0.9), targets], axis=1)
    # plus one target above and one below the predicted range
    q = np.vstack([q, [0.8, 0.9, hi_lo[0] * 1.5], [0.8, 0.9, hi_lo[1] * 0.5]])
    got = net.invert_kappa(q, 0.0, 0.95)
    for i in range(9):
        ref = M.invert_kappa(th64, norm, 0.8, 0.9, targets[i])
        assert got[i] == pytest.approx(ref, abs=1e-4)
        # and the predicted sigma at the answer is the target
        s = M.forward(th64, np.array([[0.8, got[i], 0.9]]), norm)[0][0, 0]
        assert s == pytest.approx(targets[i], rel=2e-3)
    assert np.isnan(got[9]) and np.isnan(got[10])
    net.close()


def test_argument_errors(lbm):
    net = lbm.MLP(10)
    with pytest.raises(lbm.LBError) as e:
        net.loss_grad()
    assert e.value.status == lbm.LB_EINVAL
    x, y = I.mlp_random_data(11, seed=1)
    with pytest.raises(lbm.LBError):
        net.set_data(x, y)                       # more samples than max_samples
    y[3, 0] = 0.0
    with pytest.raises(lbm.LBError):
        net.set_data(x[:10], y[:10])             # sigma <= 0 cannot be log-transformed
    y[3, 0] = np.nan
    with pytest.raises(lbm.LBError):
        net.set_data(x[:10], y[:10])
    with pytest.raises(lbm.LBError):
        net.invert_kappa(np.zeros((1, 3)), 0.5, 0.5)
    with pytest.raises(lbm.LBError):
        net.invert_kappa(np.zeros((1, 3)), 0.5, 1.0)          # ln(1 - kappa) undefined
    with pytest.raises(lbm.LBError):
        net.forward(np.array([[1.0, 0.2, 0.9]]))               # T = T_c
    xb = x[:10].copy()
    xb[0, 1] = 1.0
    with pytest.raises(lbm.LBError):
        net.set_data(xb, np.abs(I.mlp_random_data(10, seed=2)[1]))
    with pytest.raises(lbm.LBError):
        net.set_norm([np.zeros(3), np.zeros(3), np.zeros(3), np.ones(3)])
    net.set_data(x[:10], np.abs(I.mlp_random_data(10, seed=2)[1]))
    with pytest.raises(lbm.LBError):
        net.train(5, -1.0)
    net.close()
