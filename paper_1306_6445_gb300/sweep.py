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
                       tick: int = TICK, extensions: int = 2, tol: float = 0.01):
    """Advance a batch whose lattices have budgets[i] steps each (multiples of `window`,
    starting at step 0), retiring every lattice (lb_batch_set_active) once it is done, so
    the work of a lattice is proportional to its own step count. The Laplace reading of
    lattice i is averaged over the `window` steps before check_at x its budget (rounded to
    a window) and over the `window` steps before its budget; the lattice is converged when
    the two agree within `tol`. If they do not, it runs on for half its budget more (up to
    `extensions` times) and its last two readings are compared again.

    Returns a dict of arrays: theta (the last reading), theta_check (the one before),
    rho_l, rho_v (last reading), failed, converged, steps (each lattice's total)."""
    budgets = np.asarray(budgets, dtype=np.int64)
    radii = np.asarray(radii, dtype=np.float64)
    n = len(budgets)
    if np.any(budgets % window) or np.any(budgets < 4 * window):
        raise ValueError("budgets must be multiples of the window, at least four windows")
    checks = np.round(check_at * budgets / window).astype(np.int64) * window
    checks = np.clip(checks, window, budgets - window)
    ext = np.maximum((budgets // 2) // window * window, window)
    end = checks.copy()                    # end of each lattice's next reading window
    last_end = budgets.copy()              # step at which the lattice is checked next
    acc = np.zeros((n, 3))
    cnt = np.zeros(n)
    prev = np.full((n, 3), np.nan)         # the reading before the current one
    cur = np.full((n, 3), np.nan)
    left = np.full(n, extensions)
    failed = np.zeros(n, dtype=bool)
    conv = np.zeros(n, dtype=bool)
    active = np.ones(n, dtype=bool)
    steps = np.zeros(n, dtype=np.int64)
    s = 0
    while active.any():
        nxt = s + tick
        inw = active & (nxt > end - window) & (nxt <= end)
        if inw.any():
            b.step(tick)
            steps[active] += tick
            s = nxt
            m = b.measure(radii)
            acc[inw] += m[inw, :3]
            cnt[inw] += 1
            failed |= inw & (m[:, 7] != 0)
            fin = inw & (end == s)         # a reading window closes
            for i in np.flatnonzero(fin):
                prev[i], cur[i] = cur[i], acc[i] / cnt[i]
                acc[i], cnt[i] = 0.0, 0
                if s < last_end[i]:        # the check reading: the next one ends the budget
                    end[i] = last_end[i]
                    continue
                conv[i] = (not failed[i]) and abs(cur[i, 0] / prev[i, 0] - 1.0) < tol
                if conv[i] or failed[i] or left[i] == 0:
                    active[i] = False
                else:                      # run on and read again
                    left[i] -= 1
                    last_end[i] += ext[i]
                    end[i] = last_end[i]
            if (fin & ~active).any():      # some lattice finished in this tick
                b.set_active(active)
        else:
            # jump to the start of the next reading window of an active lattice
            starts = (end - window)[active]
            s_to = int(starts[starts > s].min()) if np.any(starts > s) else int(end[active].min())
            b.step(s_to - s)
            steps[active] += s_to - s
            s = s_to
    return {"theta": cur[:, 0], "theta_check": prev[:, 0], "rho_l": cur[:, 1],
            "rho_v": cur[:, 2], "failed": failed, "converged": conv, "steps": steps}


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
