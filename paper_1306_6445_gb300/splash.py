"""Droplet splashing on a thin liquid film (Sec. V.C): lattice set-up and the spread
radius. The update runs in the library (LB_BC_OPEN: no-slip bottom, zero-gradient open
top and sides; nu(rho) switched at a density rho_1); this module only builds the initial
state and reads the density field.

Readings (the paper gives none of these): the droplet starts `gap` lattice units above the
film with velocity (0, -U) inside it; the spread radius is the largest distance from the
impact axis of liquid (rho above the mean of the two phase densities) in the row 0.1 D
above the undisturbed film surface."""
from __future__ import annotations

import numpy as np

from . import inputs as I


def make_lattice(lbm, nx, ny, eos, G, kappa, sigma_force, D, film, U, nu_l, nu_v, rho_1,
                 rho_l, rho_v, prec="fp32", gap=2.0):
    """A set-up splash lattice: MRT rates of Sec. V.C (s_rho = s_j = 1, s_e = s_zeta = 0.8,
    s_q = 1.1), s_v from nu_l, the vapour rate from nu_v below rho_1."""
    rates = lbm.RateParams(s_rho=1.0, s_e=0.8, s_zeta=0.8, s_j=1.0, s_q=1.1,
                           s_v=1.0 / (3.0 * nu_l + 0.5))
    lat = lbm.Lattice(nx, ny, eos, G, kappa=kappa, sigma_force=sigma_force, rates=rates,
                      prec=prec, open_bc=True,
                      viscosity_switch=(rho_1, 1.0 / (3.0 * nu_v + 0.5)))
    lat.set_rho_u(*I.splash_state(nx, ny, film, 0.5 * D, gap, U, rho_l, rho_v))
    return lat


def spread_radius(rho, film, D, rho_l, rho_v):
    """r / D from a density field [ny][nx] (impact axis at nx/2)."""
    nx = rho.shape[1]
    row = rho[int(film + 0.1 * D)]
    liquid = np.flatnonzero(row > 0.5 * (rho_l + rho_v))
    return float(np.max(np.abs(liquid - 0.5 * nx)) / D) if liquid.size else 0.0
