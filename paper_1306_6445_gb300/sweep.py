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
