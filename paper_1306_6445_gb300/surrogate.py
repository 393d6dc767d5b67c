"""Surrogate of the Laplace-law sweep: fit the 3-64-64-3 network (lb_mlp_*) to batched
measurements and use it to choose kappa for a target surface tension.

The paper tunes sigma through kappa (Eq. 18) with sigma = (1 - kappa) sigma_0 to leading
order (Eq. 22); the network learns the measured map instead, so a target sigma needs no
kappa = 0 calibration run and follows the measured departure from that law. Training and
inference run in the library's kernels; this module only schedules them.
"""
from __future__ import annotations

import numpy as np

from . import inputs as I
from . import sweep

# full-batch Adam: (steps, learning rate) stages
SCHEDULE = ((4000, 3e-3), (4000, 1e-3), (4000, 3e-4), (4000, 1e-4))


def fit(lbm, x, y, seed: int = 1306, schedule=SCHEDULE):
    """x: n x 3 (T/T_c, kappa, tau_v), y: n x 3 (sigma, rho_l, rho_v) with every entry
    positive. Returns (network, list of the loss after each stage)."""
    x = np.asarray(x, dtype=np.float32)
    y = np.asarray(y, dtype=np.float32)
    net = lbm.MLP(max(1, x.shape[0]))
    net.set_params(I.mlp_init(seed))
    net.set_data(x, y)
    losses = [net.train(steps, lr) for steps, lr in schedule]
    return net, losses


def choose_kappa(net, t_over_tc, tau_v, sigma_target, kappa_range=(0.0, 0.95)):
    """kappa for each target (arrays broadcast together); NaN where the target lies
    outside the network's sigma over kappa_range."""
    t, tau, s = np.broadcast_arrays(np.asarray(t_over_tc, dtype=np.float64),
                                    np.asarray(tau_v, dtype=np.float64),
                                    np.asarray(sigma_target, dtype=np.float64))
    q = np.stack([t.ravel(), tau.ravel(), s.ravel()], axis=1)
    return net.invert_kappa(q, *kappa_range).astype(np.float64).reshape(t.shape)


def tune_kappa(lbm, net, t_over_tc, tau_v, sigma_target, tol: float = 0.02,
               max_rounds: int = 4, **laplace_kw):
    """Choose kappa for each target and verify it with a plain Laplace run (the check).

    Round 0 takes the network's kappa (NaN targets go straight to the fallback) and
    measures sigma at it, all points in one batched run. Points that miss by more than
    `tol` fall back to the Laplace-law sweep: a kappa = 0 run gives sigma_0 and the law
    kappa = 1 - sigma*/sigma_0 (Eq. 22); later rounds correct kappa with the measured
    ln sigma against ln(1 - kappa) (secant through the two measurements nearest the
    target, or the law's unit slope from one), one batched run
    per round. Returns dict(kappa, sigma, rel_err, runs) with runs = Laplace runs spent
    per point (1 when the network alone was right)."""
    t = np.atleast_1d(np.asarray(t_over_tc, dtype=np.float64))
    tau = np.broadcast_to(np.asarray(tau_v, dtype=np.float64), t.shape).copy()
    target = np.broadcast_to(np.asarray(sigma_target, dtype=np.float64), t.shape).copy()
    n = t.size
    kappa = choose_kappa(net, t, tau, target) if net is not None else np.full(n, np.nan)
    sigma = np.full(n, np.nan)
    runs = np.zeros(n, dtype=int)
    have = ~np.isnan(kappa)
    if have.any():
        m = sweep_points(lbm, t[have], kappa[have], tau[have], **laplace_kw)
        sigma[have] = m
        runs[have] += 1
    history = [[] for _ in range(n)]        # (ln(1 - kappa), ln sigma) measured
    for i in np.flatnonzero(have):
        if sigma[i] > 0:
            history[i].append((np.log1p(-kappa[i]), np.log(sigma[i])))
    for _ in range(max_rounds):
        miss = ~(np.abs(sigma / target - 1) <= tol)
        if not miss.any():
            break
        idx = np.flatnonzero(miss)
        need0 = [i for i in idx if not any(h[0] == 0.0 for h in history[i])]
        if need0:   # sigma_0 for the law
            s0 = sweep_points(lbm, t[need0], np.zeros(len(need0)), tau[need0], **laplace_kw)
            for i, s in zip(need0, s0):
                runs[i] += 1
                if s > 0:
                    history[i].append((0.0, np.log(s)))
        for i in idx:
            lt = np.log(target[i])
            h = sorted(history[i], key=lambda p: abs(p[1] - lt))[:2]   # nearest the target
            if not h:
                xn = 0.0
            else:
                slope = 1.0                   # the law of Eq. 22: ln sigma rises 1:1
                if len(h) == 2 and h[0][0] != h[1][0]:
                    sl = (h[0][1] - h[1][1]) / (h[0][0] - h[1][0])
                    if sl > 0:
                        slope = sl
                xn = h[0][0] + (lt - h[0][1]) / slope
            kappa[i] = float(np.clip(-np.expm1(xn), 0.0, 0.99))
        m = sweep_points(lbm, t[idx], kappa[idx], tau[idx], **laplace_kw)
        for i, s in zip(idx, m):
            runs[i] += 1
            sigma[i] = s
            if s > 0:
                history[i].append((np.log1p(-kappa[i]), np.log(s)))
    return {"kappa": kappa, "sigma": sigma, "rel_err": sigma / target - 1, "runs": runs}


def sweep_points(lbm, t, kappa, tau, **laplace_kw):
    """Measured sigma at each (T/T_c, kappa, tau_v) (NaN for a failed lattice)."""
    r = sweep.laplace_points(lbm, np.stack([t, kappa, tau], axis=1), **laplace_kw)
    s = r[:, 0].copy()
    s[r[:, 3] != 0] = np.nan
    return s
