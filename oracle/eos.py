"""Equations of state, pseudopotentials and coexistence tools (FP64, scipy).

Test infrastructure only (see ``oracle/__init__``).

Lattice units throughout: c = delta_x = delta_t = 1, c_s^2 = 1/3 (Sec. II).

Sources in the paper
--------------------
* exponential pseudopotential psi = psi0 exp(-rho0/rho), Sec. II (text after Eq. 7);
  its equation of state is p0 = rho c_s^2 + G psi^2 / 2 (Sec. III, text after Eq. 10
  with G1 = G, G2 = 0).
* EOS-based pseudopotential psi = sqrt(2 (p_EOS - rho c_s^2) / (G c^2)), Sec. II.
* Carnahan-Starling EOS: named in Sec. II and Sec. V.C; the formula used is the
  standard one, p = rho R T (1 + eta + eta^2 - eta^3) / (1 - eta)^3 - a rho^2 with
  eta = b rho / 4.
* piecewise-linear EOS, Eq. 23 (Sec. V.A), parameters theta_V = 0.49 c_s^2,
  theta_M = -0.06 c_s^2, theta_L = c_s^2, rho_1 = 1.49, rho_2 = 94.65.
* Maxwell construction (equal area in 1/rho), Sec. II.
* mechanical-stability condition, Eq. 16 (Sec. III.A).
* flat-interface surface tension from the pressure tensor of Eq. 22 (Sec. IV).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy import integrate, optimize

CS2 = 1.0 / 3.0  # c_s^2 of D2Q9 in lattice units


class DomainError(ValueError):
    """psi^2 < 0: the EOS left the branch where the pseudopotential is real."""


@dataclass(frozen=True)
class EOS:
    """Equation of state / pseudopotential choice.

    kind = "cs"        Carnahan-Starling with a, b, R, T
    kind = "exp"       psi = psi0 exp(-rho0 / rho)
    kind = "piecewise" Eq. 23 with theta_v, theta_m, theta_l, rho1, rho2
    """

    kind: str
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    T: float = 0.0
    psi0: float = 4.0
    rho0: float = 200.0
    theta_v: float = 0.49 * CS2
    theta_m: float = -0.06 * CS2
    theta_l: float = CS2
    rho1: float = 1.49
    rho2: float = 94.65


def colosqui_eos() -> EOS:
    """The piecewise-linear EOS of Eq. 23 with the parameters of Sec. V.A."""
    return EOS(kind="piecewise")


# --------------------------------------------------------------------------------------
# p_EOS(rho) and its derivative
# --------------------------------------------------------------------------------------

def p_eos(rho, eos: EOS, G: float):
    """Bulk pressure p0(rho).

    For the EOS-based potential this is the prescribed p_EOS; for the exponential
    potential it is rho c_s^2 + G psi^2 / 2 (Sec. III, with G1 = G, G2 = 0)."""
    rho = np.asarray(rho, dtype=np.float64)
    if eos.kind == "cs":
        eta = eos.b * rho / 4.0
        return rho * eos.R * eos.T * (1 + eta + eta**2 - eta**3) / (1 - eta) ** 3 - eos.a * rho**2
    if eos.kind == "exp":
        psi = eos.psi0 * np.exp(-eos.rho0 / rho)
        return rho * CS2 + 0.5 * G * psi**2
    if eos.kind == "piecewise":
        r1, r2 = eos.rho1, eos.rho2
        low = rho * eos.theta_v
        mid = r1 * eos.theta_v + (rho - r1) * eos.theta_m
        high = r1 * eos.theta_v + (r2 - r1) * eos.theta_m + (rho - r2) * eos.theta_l
        return np.where(rho <= r1, low, np.where(rho < r2, mid, high))
    raise ValueError(f"unknown EOS kind {eos.kind!r}")


def dp_drho(rho, eos: EOS, G: float):
    """d p0 / d rho, written out from the formulas of ``p_eos``."""
    rho = np.asarray(rho, dtype=np.float64)
    if eos.kind == "cs":
        eta = eos.b * rho / 4.0
        # d/d rho [rho Z(eta)] with Z = (1+eta+eta^2-eta^3)/(1-eta)^3 equals
        # (1 + 4 eta + 4 eta^2 - 4 eta^3 + eta^4) / (1 - eta)^4.
        g = (1 + 4 * eta + 4 * eta**2 - 4 * eta**3 + eta**4) / (1 - eta) ** 4
        return eos.R * eos.T * g - 2 * eos.a * rho
    if eos.kind == "exp":
        psi = eos.psi0 * np.exp(-eos.rho0 / rho)
        return CS2 + G * psi**2 * eos.rho0 / rho**2
    if eos.kind == "piecewise":
        return np.where(rho <= eos.rho1, eos.theta_v,
                        np.where(rho < eos.rho2, eos.theta_m, eos.theta_l))
    raise ValueError(f"unknown EOS kind {eos.kind!r}")


# --------------------------------------------------------------------------------------
# pseudopotential
# --------------------------------------------------------------------------------------

def psi_of_rho(rho, eos: EOS, G: float):
    """Interaction potential psi(rho) of Sec. II.

    exp:        psi = psi0 exp(-rho0 / rho)
    cs, piecewise:  psi = sqrt(2 (p_EOS - rho c_s^2) / (G c^2)), c = 1.
    Raises DomainError where the square root argument is negative."""
    rho = np.asarray(rho, dtype=np.float64)
    if eos.kind == "exp":
        return eos.psi0 * np.exp(-eos.rho0 / rho)
    arg = 2.0 * (p_eos(rho, eos, G) - rho * CS2) / G
    if np.any(arg < 0) or np.any(~np.isfinite(arg)):
        raise DomainError("psi^2 < 0 (or non-finite): density outside the EOS branch")
    return np.sqrt(arg)


def dpsi_drho(rho, eos: EOS, G: float):
    """d psi / d rho.

    exp:  psi rho0 / rho^2.
    EOS-based: from psi^2 = 2 (p - rho/3) / G, 2 psi psi' = 2 (p' - 1/3) / G."""
    rho = np.asarray(rho, dtype=np.float64)
    psi = psi_of_rho(rho, eos, G)
    if eos.kind == "exp":
        return psi * eos.rho0 / rho**2
    return (dp_drho(rho, eos, G) - CS2) / (G * psi)


# --------------------------------------------------------------------------------------
# Carnahan-Starling critical point
# --------------------------------------------------------------------------------------

def cs_critical(a: float = 1.0, b: float = 4.0, R: float = 1.0):
    """(T_c, rho_c) of the Carnahan-Starling EOS from dp/drho = d2p/drho2 = 0.

    With eta = b rho / 4 and h(eta) = eta Z(eta), p = (4 R T / b) h(eta) - a (4 eta / b)^2.
    The two conditions give R T = 8 a / (b h''(eta)) and h'(eta) = eta h''(eta);
    the second is solved for eta in (0, 1)."""
    P = np.polynomial.Polynomial
    num1 = P([1, 4, 4, -4, 1])          # h'(eta) numerator
    den1 = P([1, -1]) ** 4              # h'(eta) denominator (1 - eta)^4

    def h1(eta):
        return num1(eta) / den1(eta)

    def h2(eta):  # quotient rule on h'
        return (num1.deriv()(eta) * den1(eta) - num1(eta) * den1.deriv()(eta)) / den1(eta) ** 2

    eta_c = optimize.brentq(lambda e: h1(e) - e * h2(e), 1e-6, 0.9, xtol=1e-15, rtol=1e-15)
    T_c = 8.0 * a / (b * R * h2(eta_c))
    rho_c = 4.0 * eta_c / b
    return float(T_c), float(rho_c)


def cs_eos(T_over_Tc: float, a: float = 1.0, b: float = 4.0, R: float = 1.0) -> EOS:
    Tc, _ = cs_critical(a, b, R)
    return EOS(kind="cs", a=a, b=b, R=R, T=T_over_Tc * Tc)


# --------------------------------------------------------------------------------------
# coexistence: Maxwell construction and the mechanical-stability condition (Eq. 16)
# --------------------------------------------------------------------------------------

def _spinodals(eos: EOS, G: float, rho_max: float):
    """(rho_a, rho_b): local maximum and local minimum of p0(rho) in (0, rho_max)."""
    if eos.kind == "piecewise":
        return eos.rho1, eos.rho2
    grid = np.linspace(rho_max * 1e-4, rho_max, 20001)
    dp = dp_drho(grid, eos, G)
    sign_change = np.nonzero(np.diff(np.sign(dp)))[0]
    if len(sign_change) < 2:
        raise ValueError("EOS has no van der Waals loop in the scanned range")
    i, j = sign_change[0], sign_change[1]
    ra = optimize.brentq(lambda r: dp_drho(r, eos, G), grid[i], grid[i + 1], xtol=1e-15)
    rb = optimize.brentq(lambda r: dp_drho(r, eos, G), grid[j], grid[j + 1], xtol=1e-15)
    return ra, rb


def _rho_max(eos: EOS) -> float:
    if eos.kind == "cs":
        return 0.999 * 4.0 / eos.b      # eta < 1
    if eos.kind == "exp":
        return 10.0 * eos.rho0
    return 10.0 * eos.rho2


def _branch_roots(p_b, eos, G, ra, rb, rho_max):
    f = lambda r: float(p_eos(r, eos, G)) - p_b  # noqa: E731
    lo = ra * 1e-3
    while f(lo) > 0 and lo > 1e-300:
        lo *= 1e-3
    rho_v = optimize.brentq(f, lo, ra, xtol=1e-15, rtol=1e-15, maxiter=500)
    rho_l = optimize.brentq(f, rb, rho_max, xtol=1e-15, rtol=1e-15, maxiter=500)
    return rho_v, rho_l


def _coexistence(eos: EOS, G: float, weight):
    """Solve p0(rho_V) = p0(rho_L) = p_b and int_{rho_V}^{rho_L} (p_b - p0) weight drho = 0."""
    rho_max = _rho_max(eos)
    ra, rb = _spinodals(eos, G, rho_max)
    p_hi = float(p_eos(ra, eos, G))
    p_lo = max(float(p_eos(rb, eos, G)), 1e-9 * p_hi)
    pts = [eos.rho1, eos.rho2] if eos.kind == "piecewise" else None

    def area(p_b):
        rv, rl = _branch_roots(p_b, eos, G, ra, rb, rho_max)
        kw = {"points": [x for x in pts if rv < x < rl]} if pts else {}
        val, _ = integrate.quad(lambda r: (p_b - float(p_eos(r, eos, G))) * weight(r),
                                rv, rl, limit=400, epsabs=0, epsrel=1e-12, **kw)
        return val

    span = p_hi - p_lo
    lo, hi = p_lo + 1e-12 * span, p_hi - 1e-12 * span
    if np.sign(area(lo)) == np.sign(area(hi)):
        raise ValueError("no coexistence solution: the area condition has no root between the "
                         "spinodal pressures")
    p_b = optimize.brentq(area, lo, hi, xtol=1e-16, rtol=1e-15, maxiter=500)
    rv, rl = _branch_roots(p_b, eos, G, ra, rb, rho_max)
    return rv, rl, p_b


def maxwell(eos: EOS, G: float = -1.0):
    """Maxwell equal-area construction (Sec. II): int (p_b - p0) / rho^2 drho = 0.

    Returns (rho_V, rho_L, p_b)."""
    return _coexistence(eos, G, lambda r: 1.0 / r**2)


def mechanical_stability(eos: EOS, G: float, eps: float = 0.0):
    """Coexistence densities of the pseudopotential LB model from Eq. 16:

        int_{rho_V}^{rho_L} (p_b - rho c_s^2 - G psi^2 / 2) psi' / psi^(1+eps) drho = 0,

    with rho c_s^2 + G psi^2 / 2 = p0 for both potentials. eps = 0 for the
    single-range force of Eq. 7 with the forcing of Eq. 5. Returns (rho_V, rho_L, p_b)."""
    def weight(r):
        psi = float(psi_of_rho(r, eos, G))
        return float(dpsi_drho(r, eos, G)) / psi ** (1.0 + eps)
    return _coexistence(eos, G, weight)


# --------------------------------------------------------------------------------------
# flat-interface surface tension implied by Eq. 22
# --------------------------------------------------------------------------------------

def flat_surface_tension(eos: EOS, G: float, kappa: float, coexistence=None) -> float:
    """Surface tension of a flat interface in the continuum limit of Eq. 22.

    For a flat interface with normal n, Eq. 22 gives
        P_nn = p0 + (G/4) psi psi''       (independent of kappa),
        P_tt = p0 + (G/12)(1 + 2 kappa) psi psi'',
    so theta = int (P_nn - P_tt) dn = -(G/6)(1 - kappa) int psi_n^2 dn after one
    integration by parts. Mechanical equilibrium P_nn = p_b gives
        psi_n^2(rho) = (8/G) int_{rho_V}^{rho} (p_b - p0) psi' / psi drho',
    and int psi_n^2 dn = int_{rho_V}^{rho_L} sqrt(psi_n^2) psi'(rho) drho.
    The bulk densities are those of Eq. 16 with eps = 0 unless given."""
    if coexistence is None:
        coexistence = mechanical_stability(eos, G, 0.0)
    rv, rl, p_b = coexistence
    pts = [x for x in ([eos.rho1, eos.rho2] if eos.kind == "piecewise" else []) if rv < x < rl]

    def inner_integrand(r):
        return (p_b - float(p_eos(r, eos, G))) * float(dpsi_drho(r, eos, G)) / float(
            psi_of_rho(r, eos, G))

    def psi_n_sq(r):
        kw = {"points": [x for x in pts if x < r]} if pts and any(x < r for x in pts) else {}
        val, _ = integrate.quad(inner_integrand, rv, r, limit=400, epsabs=0, epsrel=1e-12, **kw)
        return max(8.0 / G * val, 0.0)

    kw = {"points": pts} if pts else {}
    total, _ = integrate.quad(lambda r: np.sqrt(psi_n_sq(r)) * float(dpsi_drho(r, eos, G)),
                              rv, rl, limit=400, epsabs=0, epsrel=1e-10, **kw)
    return -(G / 6.0) * (1.0 - kappa) * total
