"""FP64 reference of the surrogate network (plain numpy), for parity tests of the CUDA
training and inference kernels.

Test infrastructure only (see ``oracle/__init__``).

Network (the surrogate of the batched Laplace sweep): inputs (T/T_c, kappa, tau_v),
outputs (theta, rho_l, rho_v). The inputs enter as the features
(ln(1 - T/T_c), ln(1 - kappa), tau_v), standardised with given means / scales; the outputs
are learnt in the space (log theta, rho_l, log rho_v), standardised the same way. Two hidden layers of width 64 with GELU, GELU(x) = x Phi(x) = x/2 (1 + erf(x/sqrt 2)).
Weights are used as BF16 (round to nearest even of the FP32 master copy), activations
and sums in FP64 here (FP32 on the GPU).

Parameter vector layout (FP32 master copy, 4611 values):
  W1[64][3], b1[64], W2[64][64], b2[64], W3[3][64], b3[3]    (row-major, out x in)
Loss: mean over samples and the three outputs of the squared error in the standardised
output space. Optimiser: Adam (Kingma & Ba) with beta1, beta2, eps, bias correction.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

H = 64
SIZES = [(H, 3), (H,), (H, H), (H,), (3, H), (3,)]
N_PARAMS = sum(int(np.prod(s)) for s in SIZES)


def unpack(theta):
    out, k = [], 0
    for s in SIZES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[k:k + n], dtype=np.float64).reshape(s))
        k += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def bf16_round(x):
    """Round FP32 values to BF16 (8 exponent bits, 7 fraction bits), nearest even,
    returned as FP32: keep the top 16 bits of the FP32 pattern after adding half an ulp
    of the dropped part (plus the tie-to-even bit)."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def features(x):
    """(T/T_c, kappa, tau_v) -> (ln(1 - T/T_c), ln(1 - kappa), tau_v)."""
    x = np.asarray(x, dtype=np.float64)
    return np.stack([np.log1p(-x[:, 0]), np.log1p(-x[:, 1]), x[:, 2]], axis=1)


def to_net_targets(y):
    """(theta, rho_l, rho_v) -> (log theta, rho_l, log rho_v)."""
    y = np.asarray(y, dtype=np.float64)
    return np.stack([np.log(y[:, 0]), y[:, 1], np.log(y[:, 2])], axis=1)


def from_net_outputs(o):
    return np.stack([np.exp(o[:, 0]), o[:, 1], np.exp(o[:, 2])], axis=1)


def normalisation(x, y):
    """Means and scales (population standard deviation; 1 where it is no more than 1e-9 of
    the mean's magnitude, i.e. a constant column up to rounding) of the input features and
    of the transformed targets, returned as (in_mean, in_scale, out_mean, out_scale)."""
    x = features(x)
    t = to_net_targets(y)

    def ms(a):
        m = a.mean(axis=0)
        s = np.sqrt(((a - m) ** 2).mean(axis=0))
        return m, np.where((s > 0) & (s > 1e-9 * np.abs(m)), s, 1.0)

    return (*ms(x), *ms(t))


def forward(theta, x, norm, bf16=True):
    """Returns (predictions (theta, rho_l, rho_v), standardised outputs, cache)."""
    W1, b1, W2, b2, W3, b3 = unpack(bf16_round(theta) if bf16 else theta)
    in_m, in_s, out_m, out_s = (np.asarray(v, dtype=np.float64) for v in norm)
    xn = (features(x) - in_m) / in_s
    z1 = xn @ W1.T + b1
    a1 = gelu(z1)
    z2 = a1 @ W2.T + b2
    a2 = gelu(z2)
    o = a2 @ W3.T + b3
    y = from_net_outputs(o * out_s + out_m)
    return y, o, (xn, z1, a1, z2, a2, W1, W2, W3)


def loss_and_grad(theta, x, y, norm, bf16=True):
    """Mean squared error in the standardised output space and its gradient with respect
    to the (BF16-rounded) parameters, by the chain rule."""
    in_m, in_s, out_m, out_s = (np.asarray(v, dtype=np.float64) for v in norm)
    _, o, (xn, z1, a1, z2, a2, W1, W2, W3) = forward(theta, x, norm, bf16)
    t = (to_net_targets(y) - out_m) / out_s
    n = x.shape[0]
    r = o - t
    loss = np.mean(r * r)
    do = 2.0 * r / (n * 3)
    gW3 = do.T @ a2
    gb3 = do.sum(axis=0)
    da2 = do @ W3
    dz2 = da2 * gelu_grad(z2)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(axis=0)
    da1 = dz2 @ W2
    dz1 = da1 * gelu_grad(z1)
    gW1 = dz1.T @ xn
    gb1 = dz1.sum(axis=0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam_step(theta, m, v, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def invert_kappa(theta, norm, t_over_tc, tau, target, lo=0.0, hi=0.95, iters=40):
    """Bisection for kappa with predicted theta(T, kappa, tau) = target (theta decreases
    with kappa, Eq. 22); NaN when the target is outside [theta(hi), theta(lo)]."""
    def th(k):
        return forward(theta, np.array([[t_over_tc, k, tau]]), norm)[0][0, 0]

    if not (th(lo) >= target >= th(hi)):
        return float("nan")
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if th(mid) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
