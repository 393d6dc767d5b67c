"""Laplace-law measurements of many droplets at once (batched lattices), the training data
and the check of the surrogate network.

Each point (T/T_c, kappa, tau_v) becomes one periodic side x side lattice of the
Carnahan-Starling fluid (a = 1, b = 4, R = 1, G = -1, sigma_F = 0.087 in Eq. 8, MRT rates
s_e = s_zeta = 0.8, s_q = 1.1, s_v = 1/tau_v) holding a centred droplet of the given radius
between the Maxwell coexistence densities. All lattices advance together through
lb_batch_step; the surface tension is sigma = (p_in - p_out) R (Laplace law, Sec. V.A),
measured on the GPU by lb_batch_measure and averaged over the last `window` steps (one
reading every 64 steps) so that the residual acoustic oscillation of the periodic box
averages out. Everything here is orchestration: the work runs in the library.
"""
from __future__ import annotations

import numpy as np

from . import inputs as I

SIGMA_FORCE = 0.087
G = -1.0


def laplace_points(lbm, points, side: int = 128, radius: float | None = None,
                   steps: int = 24000, window: int = 2048, prec: str = "fp32",
                   autotune: bool = True):
    """points: n x 3 array of (T/T_c, kappa, tau_v). Returns n x 4 float64 array of
    (sigma, rho_l, rho_v, failed) with rho_l / rho_v the mean densities inside / outside
    the droplet (the measurement regions of lb_batch_measure)."""
    pts = np.atleast_2d(np.asarray(points, dtype=np.float64))
    n = pts.shape[0]
    if radius is None:
        radius = 0.25 * side
    if window % 64 or window > steps:
        raise ValueError("window must be a multiple of 64 and at most steps")
    descs, init = [], []
    for t, kappa, tau in pts:
        eos = lbm.cs_eos(float(t))
        rv, rl, _ = lbm.lb_maxwell(eos, G)
        descs.append(lbm.LatticeDesc(side, side, eos, G, kappa=float(kappa),
                                     sigma_force=SIGMA_FORCE,
                                     rates=lbm.RateParams(s_v=1.0 / float(tau))))
        init.append((rl, rv))
    b = lbm.Batch(descs, prec=prec)
    try:
        for i, (rl, rv) in enumerate(init):
            b.set_rho_u(i, I.droplet_density(side, side, radius, rl, rv))
        if autotune:
            b.autotune(2)   # timed on these states, which it restores
        radii = np.full(n, float(radius))
        b.step(steps - window)
        acc = np.zeros((n, 3))
        failed = np.zeros(n, dtype=bool)
        k = window // 64
        for _ in range(k):
            b.step(64)
            m = b.measure(radii)
            acc += m[:, :3]
            failed |= m[:, 7] != 0
        out = np.empty((n, 4))
        out[:, :3] = acc / k
        out[:, 3] = failed
        return out
    finally:
        b.close()


def linear_law_kappa(sigma_target: float, sigma0: float) -> float:
    """The surrogate-free choice: kappa = 1 - sigma*/sigma_0 from a kappa = 0 measurement
    (the leading-order law sigma = (1 - kappa) sigma_0 of Eq. 22)."""
    return 1.0 - sigma_target / sigma0


def training_points(n: int, seed: int = 1306) -> np.ndarray:
    """(T/T_c, kappa, tau_v) drawn like the batched sweep: U[0.65, 0.95] x U[0, 0.95] x
    U[0.6, 1.2]."""
    d = I.batch_draws(n, seed)
    return np.array([[e["t_over_tc"], e["kappa"], e["tau_v"]] for e in d])


# ---- converged sweeps of lattices of uneven size ------------------------------------------

TICK = 64         # readings are taken every TICK steps
WINDOW = 2048     # a converged reading averages the last WINDOW steps (32 readings)


def step_budget(side: int, per_site2: float = 0.5, least: int = 8192) -> int:
    """Steps a side x side droplet needs to converge: the slowest acoustic mode of the
    periodic box damps at a rate proportional to 1/side^2, so the budget grows as side^2
    (0.5 side^2 measured enough for the Laplace reading of the 64..512 sweep to settle
    within 1 %), at least `least`, rounded up to a multiple of WINDOW."""
    n = max(least, int(np.ceil(per_site2 * side * side)))
    return int(-(-n // WINDOW) * WINDOW)


def converged_readings(b, budgets, radii, check_at: float = 0.75, window: int = WINDOW,
                       tick: int = TICK):
    """Advance a batch whose lattices have budgets[i] steps each (multiples of `window`,
    starting at step 0), retiring every lattice (lb_batch_set_active) once it has taken its
    budget, so the work of a lattice is proportional to its own budget. The Laplace reading
    of lattice i is averaged over the `window` steps before its budget (B) and over the
    `window` steps before check_at x its budget (A, rounded to a window); the lattice counts
    as converged when A and B differ by less than 1 %.

    Returns a dict of arrays: theta (B), theta_check (A), rho_l, rho_v (B), failed,
    converged."""
    budgets = np.asarray(budgets, dtype=np.int64)
    radii = np.asarray(radii, dtype=np.float64)
    n = len(budgets)
    if np.any(budgets % window) or np.any(budgets < 2 * window):
        raise ValueError("budgets must be multiples of the window, at least two windows")
    checks = np.maximum(np.round(check_at * budgets / window).astype(np.int64) * window, window)
    checks = np.minimum(checks, budgets - window)
    win = [(checks - window, checks), (budgets - window, budgets)]
    acc = np.zeros((n, 2, 3))
    cnt = np.zeros((n, 2))
    failed = np.zeros(n, dtype=bool)
    active = np.ones(n, dtype=bool)
    s = 0
    while active.any():
        nxt = s + tick
        inw = [active & (nxt > lo) & (nxt <= hi) for lo, hi in win]
        if inw[0].any() or inw[1].any():
            b.step(tick)
            s = nxt
            m = b.measure(radii)
            for w in range(2):
                acc[inw[w], w] += m[inw[w], :3]
                cnt[inw[w], w] += 1
            failed |= (inw[0] | inw[1]) & (m[:, 7] != 0)
        else:
            # jump to the next window start or budget of an active lattice
            marks = np.concatenate([win[0][0][active], win[1][0][active], budgets[active]])
            s_to = int(marks[marks > s].min())
            b.step(s_to - s)
            s = s_to
        done = active & (budgets <= s)
        if done.any():
            active &= ~done
            b.set_active(active)
    theta = acc[:, 1, 0] / np.maximum(cnt[:, 1], 1)
    theta_a = acc[:, 0, 0] / np.maximum(cnt[:, 0], 1)
    conv = (~failed) & (np.abs(theta / theta_a - 1.0) < 0.01)
    return {"theta": theta, "theta_check": theta_a,
            "rho_l": acc[:, 1, 1] / np.maximum(cnt[:, 1], 1),
            "rho_v": acc[:, 1, 2] / np.maximum(cnt[:, 1], 1),
            "failed": failed, "converged": conv}


def converged_single(lat, budget: int, radius: float, check_at: float = 0.75,
                     window: int = WINDOW, tick: int = TICK):
    """converged_readings for one lattice run on its own (lb_step, lb_measure_droplet):
    returns (theta, theta_check)."""
    check = min(max(int(round(check_at * budget / window)) * window, window), budget - window)
    out = []
    done = 0
    for end in (check, budget):
        lat.step(end - window - done)
        acc = 0.0
        for _ in range(window // tick):
            lat.step(tick)
            acc += lat.measure_droplet(radius)["theta"]
        done = end
        out.append(acc / (window // tick))
    return out[1], out[0]
