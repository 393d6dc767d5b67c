"""Shared helpers for the tests: map the product's parameters onto the oracle's."""
import numpy as np

from oracle import eos as OE
from oracle import lattice as OL


def oracle_params(eos, G, kappa, sigma_force, rates, walls_y=False, open_bc=False,
                  visc_switch=None) -> OL.Params:
    """Product EOSParams / RateParams -> oracle Params (same numbers, separate code)."""
    oe = OE.EOS(kind=eos.kind, a=eos.a, b=eos.b, R=eos.R, T=eos.T, psi0=eos.psi0,
                rho0=eos.rho0, theta_v=eos.theta_v, theta_m=eos.theta_m, theta_l=eos.theta_l,
                rho1=eos.rho1, rho2=eos.rho2)
    r = OL.Rates(s_rho=rates.s_rho, s_e=rates.s_e, s_zeta=rates.s_zeta, s_j=rates.s_j,
                 s_q=rates.s_q, s_v=rates.s_v)
    return OL.Params(eos=oe, G=G, kappa=kappa, sigma_force=sigma_force, rates=r, walls_y=walls_y,
                     open_bc=open_bc, visc_switch=visc_switch)


def window(f, x, y, walls_y, half=2):
    """The (2*half+1)^2 neighbourhood of site (x, y) from f[9, ny, nx], periodic in x;
    in y periodic, or (walls) clipped to the lattice. Returns (sub, cx, cy, sub_walls):
    the site's position inside `sub`, and whether `sub` must be treated as walled."""
    _, ny, nx = f.shape
    xs = [(x + d) % nx for d in range(-half, half + 1)]
    if not walls_y:
        ys = [(y + d) % ny for d in range(-half, half + 1)]
        return f[:, ys][:, :, xs], half, half, False
    y0 = max(0, y - half)
    y1 = min(ny, y + half + 1)
    sub = f[:, y0:y1][:, :, xs]
    # a window that does not reach a wall sees fake walls at its ends, which are more than
    # `half` rows from the centre and therefore do not influence it
    return sub, half, y - y0, True


def rel_err(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max()
                 / np.abs(np.asarray(b, np.float64)).max())


def zero_crossings(ts, ys, half=2000.0):
    """Times where ys changes sign, each from a least-squares line through the samples
    within `half` steps of the sign change (the mode amplitude carries small acoustic
    ripples); sign changes closer than 2 half to the previous one count once."""
    out = []
    for i in range(len(ys) - 1):
        if ys[i] * ys[i + 1] < 0:
            tc = 0.5 * (ts[i] + ts[i + 1])
            if out and tc - out[-1] < 2.0 * half:
                continue
            s = np.abs(ts - tc) <= half
            b, a = np.polyfit(ts[s] - tc, ys[s], 1)
            out.append(tc - a / b)
    return out
