"""Droplet splashing on a thin liquid film (Sec. V.C): lattice set-up and the spread
radius. The update runs in the library (LB_BC_OPEN: no-slip bottom, zero-gradient open
top and sides; nu(rho) switched at a density rho_1); this module only builds the initial
state and reads the density field.

Readings (the paper gives none of these):
  * start: the droplet moves down at U and has already entered the film by t0 D
    (t0 = 0.05), i.e. the run starts at t* = t0 after the first contact, so no vapour
    layer is trapped between the droplet and the film; t* = t0 + U t / D;
  * spread radius: the distance from the impact axis (x = nx/2) to the outer edge of the
    liquid that is connected to the film through liquid (rho above the mean of the two
    phase densities, 4-neighbour connectivity), in the row 0.1 D above the undisturbed
    film; the edge is placed between the last liquid site and the next one by linear
    interpolation of rho. Detached secondary droplets do not count."""
from __future__ import annotations

import numpy as np
from scipy import ndimage

from . import inputs as I

T0 = 0.05   # t* at the start of a run (the droplet has entered the film by T0 D)


def make_lattice(lbm, nx, ny, eos, G, kappa, sigma_force, D, film, U, nu_l, nu_v, rho_1,
                 rho_l, rho_v, prec="fp32", t0=T0):
    """A set-up splash lattice: MRT rates of Sec. V.C (s_rho = s_j = 1, s_e = s_zeta = 0.8,
    s_q = 1.1), s_v from nu_l, the vapour rate from nu_v below rho_1; the droplet centre
    D/2 - t0 D above the film surface."""
    rates = lbm.RateParams(s_rho=1.0, s_e=0.8, s_zeta=0.8, s_j=1.0, s_q=1.1,
                           s_v=1.0 / (3.0 * nu_l + 0.5))
    lat = lbm.Lattice(nx, ny, eos, G, kappa=kappa, sigma_force=sigma_force, rates=rates,
                      prec=prec, open_bc=True,
                      viscosity_switch=(rho_1, 1.0 / (3.0 * nu_v + 0.5)))
    lat.set_rho_u(*I.splash_state(nx, ny, film, 0.5 * D, -t0 * D, U, rho_l, rho_v))
    return lat


def steps_to(t_star, D, U, t0=T0):
    """Time steps from the start of a run to the non-dimensional time t* = t0 + U t / D."""
    return int(round((t_star - t0) * D / U))


def spread_radius(rho, film, D, rho_l, rho_v):
    """r / D from a density field [ny][nx] (impact axis at x = nx/2)."""
    ny, nx = rho.shape
    mid = 0.5 * (rho_l + rho_v)
    labels, _ = ndimage.label(rho > mid)           # 4-neighbour components of the liquid
    film_labels = np.setdiff1d(np.unique(labels[0]), [0])
    y = int(film + 0.1 * D)
    row = rho[y]
    conn = np.isin(labels[y], film_labels)
    xs = np.flatnonzero(conn)
    if xs.size == 0:
        return 0.0
    xc = 0.5 * nx
    best = 0.0
    for xo, step in ((xs.min(), -1), (xs.max(), 1)):
        edge = float(xo)
        xn = xo + step
        if 0 <= xn < nx and row[xn] < mid:        # interpolate the crossing of mid
            edge = xo + step * (row[xo] - mid) / (row[xo] - row[xn])
        best = max(best, abs(edge - xc))
    return best / D
