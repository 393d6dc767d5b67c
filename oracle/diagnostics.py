"""Measurements on lattice fields (FP64): Laplace law, flat-layer densities,
interface height and the capillary-wave dispersion relation.

Test infrastructure only (see ``oracle/__init__``).

Readings (the paper does not say how it measured):
  * bulk pressure p = rho c_s^2 + (G/2) psi^2, the isotropic part of Eq. 20;
  * p_in / rho_in: mean over sites with r < R/2; p_out / rho_out: mean over sites
    with r > R + 0.3 min(nx, ny)/2 (clipped to the lattice);
  * droplet radius from the mass, R = sqrt((sum rho - rho_out N) / (pi (rho_in - rho_out)));
  * surface tension from one radius, theta = (p_in - p_out) R (Laplace law, Sec. V.A),
    or from the slope of dp against 1/R over several radii (Fig. 3 of the paper);
  * dispersion relation read as omega^2 = theta k^3 / (rho_L + rho_V) (Eq. 24 as
    printed lost the square: the printed form is dimensionally inconsistent and
    Table 4's periods only follow from the squared form).
"""
from __future__ import annotations

import numpy as np

from .lattice import Params, pressure


def laplace(rho: np.ndarray, p: Params, center=None):
    """Laplace-law measurement on a droplet density field rho[y, x].

    Returns dict(theta, dp, R, rho_in, rho_out, p_in, p_out)."""
    ny, nx = rho.shape
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.hypot(x - center[0], y - center[1])
    pres = pressure(rho, p)
    # first pass: radius from the density midpoint estimate
    rho_in0 = rho[r < 2.0].mean()
    rho_out0 = rho[r >= r.max() - 2.0].mean()
    R0 = np.sqrt(max(rho.sum() - rho_out0 * rho.size, 0.0) / (np.pi * (rho_in0 - rho_out0)))
    inside = r < 0.5 * R0
    outside = r > R0 + 0.3 * min(nx, ny) / 2.0
    if not outside.any():
        outside = r >= r.max() - 2.0
    rho_in, rho_out = rho[inside].mean(), rho[outside].mean()
    p_in, p_out = pres[inside].mean(), pres[outside].mean()
    R = np.sqrt((rho.sum() - rho_out * rho.size) / (np.pi * (rho_in - rho_out)))
    dp = p_in - p_out
    return {"theta": dp * R, "dp": dp, "R": R, "rho_in": rho_in, "rho_out": rho_out,
            "p_in": p_in, "p_out": p_out}


def laplace_fit(dps, radii):
    """Least-squares line dp = theta / R + c over several droplets (Fig. 3).
    Returns (theta, intercept)."""
    inv = 1.0 / np.asarray(radii, dtype=np.float64)
    A = np.stack([inv, np.ones_like(inv)], axis=1)
    (theta, c), *_ = np.linalg.lstsq(A, np.asarray(dps, dtype=np.float64), rcond=None)
    return float(theta), float(c)


def slab_densities(rho: np.ndarray):
    """(rho_V, rho_L) of a lattice holding a liquid slab between two flat interfaces
    normal to y: the x-averaged profile's minimum and maximum rows."""
    prof = rho.mean(axis=1)
    return float(prof.min()), float(prof.max())


def interface_height(rho_column: np.ndarray, rho_mid: float):
    """Height y where the column crosses rho_mid going upward from the liquid
    (linear interpolation between the bracketing rows)."""
    col = np.asarray(rho_column, dtype=np.float64)
    above = col < rho_mid
    idx = int(np.argmax(above))          # first vapour row from the bottom
    if idx == 0:
        return float("nan")
    y0, y1 = idx - 1, idx
    return y0 + (col[y0] - rho_mid) / (col[y0] - col[y1])


def capillary_period(theta: float, wavelength: float, rho_l: float, rho_v: float,
                     depth_l: float | None = None, depth_v: float | None = None) -> float:
    """Period T = 2 pi / omega of a capillary wave.

    Deep fluids (Eq. 24, read with omega squared): omega^2 = theta k^3 / (rho_L + rho_V).
    Finite depths (standard capillary-wave theory, a reading for the bounded lattice):
    omega^2 = theta k^3 / (rho_L coth(k h_L) + rho_V coth(k h_V))."""
    k = 2.0 * np.pi / wavelength
    cl = 1.0 if depth_l is None else 1.0 / np.tanh(k * depth_l)
    cv = 1.0 if depth_v is None else 1.0 / np.tanh(k * depth_v)
    omega = np.sqrt(theta * k**3 / (rho_l * cl + rho_v * cv))
    return 2.0 * np.pi / omega
