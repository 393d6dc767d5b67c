"""Velocity-space twin of the update for tiny lattices (plain Python loops, long double).

Test infrastructure only (see ``oracle/__init__``).

This is a second, independent formulation of one time step, used to pin the
vectorised moment-space code in ``lattice``:

* neighbour indices are explicit modular / clamped integers per site (no np.roll);
* the equilibrium is the textbook D2Q9 polynomial
  f_eq = w_a rho [1 + 3 e.v + 4.5 (e.v)^2 - 1.5 v^2] with w = 4/9, 1/9, 1/36,
  not M^-1 m_eq;
* the Guo forcing is the textbook velocity-space term
  Fbar_a = w_a [3 (e_a - v).F + 9 (e_a.v)(e_a.F)], whose moments M Fbar are the S
  of Eq. 5; the Eq. 8 addition is put on the e and zeta moments;
* the collision is done in velocity space with explicit 9x9 matrices,
  f* = f - M^-1 Lambda M (f - f_eq) + M^-1 (I - Lambda/2) M Fbar' + M^-1 C (Eq. 1),
  where M^-1 comes from a numerical inversion in long double;
* the transformation matrix is built from polynomial definitions of its rows
  (1, 3|e|^2-4, (9|e|^4-21|e|^2+8)/2, e_x, (3|e|^2-5) e_x, e_y, (3|e|^2-5) e_y,
  e_x^2-e_y^2, e_x e_y), not typed in as a table.
"""
from __future__ import annotations

import numpy as np

from .eos import psi_of_rho

LD = np.longdouble

_E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
_OPP = {a: _E.index((-ex, -ey)) for a, (ex, ey) in enumerate(_E)}


def _w_eq(ex, ey):
    n = ex * ex + ey * ey
    return LD(4) / 9 if n == 0 else (LD(1) / 9 if n == 1 else LD(1) / 36)


def _w_int(ex, ey):
    n = ex * ex + ey * ey
    return LD(0) if n == 0 else (LD(1) / 3 if n == 1 else LD(1) / 12)


def _row_polys():
    rows = [
        lambda ex, ey, n: 1,
        lambda ex, ey, n: 3 * n - 4,
        lambda ex, ey, n: (9 * n * n - 21 * n + 8) // 2,
        lambda ex, ey, n: ex,
        lambda ex, ey, n: (3 * n - 5) * ex,
        lambda ex, ey, n: ey,
        lambda ex, ey, n: (3 * n - 5) * ey,
        lambda ex, ey, n: ex * ex - ey * ey,
        lambda ex, ey, n: ex * ey,
    ]
    mat = np.zeros((9, 9), dtype=LD)
    for k, poly in enumerate(rows):
        for a, (ex, ey) in enumerate(_E):
            mat[k, a] = poly(ex, ey, ex * ex + ey * ey)
    return mat


M_BF = _row_polys()


def _inverse(mat):
    """Gauss-Jordan inversion with partial pivoting in long double."""
    n = mat.shape[0]
    aug = np.concatenate([mat.astype(LD), np.eye(n, dtype=LD)], axis=1)
    for col in range(n):
        piv = col + int(np.argmax(np.abs(aug[col:, col])))
        aug[[col, piv]] = aug[[piv, col]]
        aug[col] /= aug[col, col]
        for r in range(n):
            if r != col:
                aug[r] -= aug[r, col] * aug[col]
    return aug[:, n:]


M_BF_INV = _inverse(M_BF)


def step(f, params):
    """One update of f[alpha, y, x] (tiny lattices only), following Eqs. 1, 4-8, 17-19."""
    nine, ny, nx = f.shape
    f = f.astype(LD)
    G = LD(params.G)
    kappa = LD(params.kappa)
    sig = LD(params.sigma_force)
    r = params.rates
    lam = np.diag(np.array([r.s_rho, r.s_e, r.s_zeta, r.s_j, r.s_q, r.s_j, r.s_q, r.s_v, r.s_v],
                           dtype=LD))
    walls = params.walls_y
    open_bc = getattr(params, "open_bc", False)
    switch = getattr(params, "visc_switch", None)

    rho = np.zeros((ny, nx), dtype=LD)
    for y in range(ny):
        for x in range(nx):
            rho[y, x] = sum(f[a, y, x] for a in range(9))
    psi = psi_of_rho(rho.astype(np.float64), params.eos, params.G).astype(LD)

    def psi_at(x, y):
        if open_bc:      # nearest lattice site outside (wall row below, open elsewhere)
            x = min(max(x, 0), nx - 1)
            y = min(max(y, 0), ny - 1)
        elif walls:
            x %= nx
            y = min(max(y, 0), ny - 1)
        else:
            x %= nx
            y %= ny
        return psi[y, x]

    collision_op = M_BF_INV @ lam @ M_BF
    force_op = M_BF_INV @ (np.eye(9, dtype=LD) - lam / 2) @ M_BF
    fstar = np.zeros_like(f)
    for y in range(ny):
        for x in range(nx):
            pc = psi[y, x]
            Fx = Fy = LD(0)
            Qxx = Qyy = Qxy = LD(0)
            for (ex, ey) in _E[1:]:
                pn = psi_at(x + ex, y + ey)
                w = _w_int(ex, ey)
                Fx += w * pn * ex
                Fy += w * pn * ey
                Qxx += w * (pn - pc) * ex * ex
                Qyy += w * (pn - pc) * ey * ey
                Qxy += w * (pn - pc) * ex * ey
            Fx *= -G * pc
            Fy *= -G * pc
            qpref = kappa * G / 2 * pc
            Qxx, Qyy, Qxy = qpref * Qxx, qpref * Qyy, qpref * Qxy

            fs = f[:, y, x]
            rh = rho[y, x]
            s_v = LD(r.s_v)
            if switch is not None and rh < LD(switch[0]):   # nu(rho), Sec. V.C
                s_v = LD(switch[1])
            lam_site = lam.copy()
            lam_site[7, 7] = lam_site[8, 8] = s_v
            collision_op = M_BF_INV @ lam_site @ M_BF
            force_op = M_BF_INV @ (np.eye(9, dtype=LD) - lam_site / 2) @ M_BF
            jx = sum(fs[a] * _E[a][0] for a in range(9))
            jy = sum(fs[a] * _E[a][1] for a in range(9))
            vx = (jx + Fx / 2) / rh
            vy = (jy + Fy / 2) / rh
            v2 = vx * vx + vy * vy
            feq = np.zeros(9, dtype=LD)
            fbar = np.zeros(9, dtype=LD)
            for a, (ex, ey) in enumerate(_E):
                ev = ex * vx + ey * vy
                feq[a] = _w_eq(ex, ey) * rh * (1 + 3 * ev + LD(4.5) * ev * ev - LD(1.5) * v2)
                eF = ex * Fx + ey * Fy
                fbar[a] = _w_eq(ex, ey) * (3 * ((ex - vx) * Fx + (ey - vy) * Fy) + 9 * ev * eF)
            # Eq. 8: the extra term is part of the moment-space forcing S (S_1 and
            # S_2 = -S_1), so like the rest of S it is scaled by (I - Lambda/2) (Eq. 2).
            extra = np.zeros(9, dtype=LD)
            if sig != 0:
                tau_e = 1 / LD(r.s_e)
                add = 12 * sig * (Fx * Fx + Fy * Fy) / (pc * pc * (tau_e - LD(0.5)))
                extra[1] = add
                extra[2] = -add
            src = np.zeros(9, dtype=LD)
            src[1] = LD(1.5) * LD(r.s_e) * (Qxx + Qyy)
            src[2] = -LD(1.5) * LD(r.s_zeta) * (Qxx + Qyy)
            src[7] = -s_v * (Qxx - Qyy)
            src[8] = -s_v * Qxy
            post = (fs - collision_op @ (fs - feq) + force_op @ fbar
                    + M_BF_INV @ ((np.eye(9, dtype=LD) - lam_site / 2) @ extra)
                    + M_BF_INV @ src)
            fstar[:, y, x] = post

    out = np.zeros_like(fstar)
    for a, (ex, ey) in enumerate(_E):
        for y in range(ny):
            for x in range(nx):
                ys, xs = y - ey, (x - ex) % nx
                if open_bc:
                    if ys < 0:                              # no-slip bottom wall
                        out[a, y, x] = fstar[_OPP[a], y, x]
                    else:                                   # open: nearest lattice site
                        out[a, y, x] = fstar[a, min(ys, ny - 1), min(max(x - ex, 0), nx - 1)]
                elif walls and not (0 <= ys < ny):
                    out[a, y, x] = fstar[_OPP[a], y, x]
                else:
                    out[a, y, x] = fstar[a, ys % ny, xs]
    return out


def run(f, params, n: int):
    for _ in range(n):
        f = step(f, params)
    return f
