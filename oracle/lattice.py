"""The D2Q9 MRT pseudopotential update with the surface-tension source term, in FP64.

Test infrastructure only (see ``oracle/__init__``).

One call of ``step`` advances f(x, t) -> f(x, t + 1) in the paper's order:

  a1  rho = sum_a f_a (Eq. 6) and psi(rho) (Sec. II)
  a2  F = -G psi(x) sum_a w_a psi(x + e_a) e_a                        (Eq. 7)
  a3  Q = kappa (G/2) psi(x) sum_a w_a [psi(x + e_a) - psi(x)] e_a e_a (Eq. 19)
  a4  rho v = sum_a e_a f_a + F/2                                     (Eq. 6)
  a5  m = M f and m_eq                                                (Eq. 3)
  a6  S with S_1 of Eq. 8 (reduces to Eq. 5 when sigma_force = 0)
  a7  C                                                               (Eq. 18)
  a8  m* = m - Lambda (m - m_eq) + (I - Lambda/2) S + C               (Eq. 17)
      f* = M^-1 m*                                                    (Sec. II, after Eq. 4)
  a9  f_a(x + e_a, t + 1) = f*_a(x, t)                                (Eq. 4)

Everything is vectorised over lattice sites with numpy; there is no blocking,
fusion or reordering of the per-site arithmetic.

Layout: f has shape (9, ny, nx), index [alpha, y, x]; x is periodic. In y the
lattice is either periodic or bounded by two no-slip walls (Sec. V.B) handled
with half-way bounce-back; at a wall the missing neighbour psi is taken equal to
the psi of the adjacent fluid row (a reading: the paper names no wall scheme).

Readings where the paper is silent:
  * velocity order e0..e8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1)
    and the standard D2Q9 transformation matrix M (rows rho, e, zeta, jx, qx, jy, qy,
    pxx, pxy), which the paper uses but does not print;
  * the interaction weights w(1) = 1/3, w(2) = 1/12 are those printed under Eq. 7.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .eos import EOS, psi_of_rho

# Discrete velocities e_alpha (Sec. II)
E = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1),
              (1, 1), (-1, 1), (-1, -1), (1, -1)], dtype=np.int64)
EX = E[:, 0]
EY = E[:, 1]
OPPOSITE = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6], dtype=np.int64)

# Interaction weights w(|e_alpha|^2) of Eq. 7: w(1) = 1/3, w(2) = 1/12.
W_INT = np.array([0.0, 1 / 3, 1 / 3, 1 / 3, 1 / 3, 1 / 12, 1 / 12, 1 / 12, 1 / 12])

# Orthogonal transformation matrix M (Sec. II; standard D2Q9 rows, a reading).
M = np.array([
    [1, 1, 1, 1, 1, 1, 1, 1, 1],            # rho
    [-4, -1, -1, -1, -1, 2, 2, 2, 2],       # e
    [4, -2, -2, -2, -2, 1, 1, 1, 1],        # zeta (varsigma)
    [0, 1, 0, -1, 0, 1, -1, -1, 1],         # j_x
    [0, -2, 0, 2, 0, 1, -1, -1, 1],         # q_x
    [0, 0, 1, 0, -1, 1, 1, -1, -1],         # j_y
    [0, 0, -2, 0, 2, 1, 1, -1, -1],         # q_y
    [0, 1, -1, 1, -1, 0, 0, 0, 0],          # p_xx
    [0, 0, 0, 0, 0, 1, -1, 1, -1],          # p_xy
], dtype=np.float64)
# M is orthogonal (rows mutually orthogonal), so M^-1 = M^T diag(1 / |row|^2).
M_INV = M.T / np.sum(M * M, axis=1)[None, :]


@dataclass(frozen=True)
class Rates:
    """Relaxation rates s = 1/tau of Lambda (Sec. II):
    Lambda = diag(s_rho, s_e, s_zeta, s_j, s_q, s_j, s_q, s_v, s_v)."""

    s_rho: float = 1.0
    s_e: float = 0.8
    s_zeta: float = 0.8
    s_j: float = 1.0
    s_q: float = 1.1
    s_v: float = 1.0 / 0.8

    def diagonal(self) -> np.ndarray:
        return np.array([self.s_rho, self.s_e, self.s_zeta, self.s_j, self.s_q,
                         self.s_j, self.s_q, self.s_v, self.s_v])

    @staticmethod
    def from_viscosity(nu: float, **kw) -> "Rates":
        """s_v from the kinematic viscosity nu = (1/s_v - 1/2) c_s^2."""
        return Rates(s_v=1.0 / (3.0 * nu + 0.5), **kw)


@dataclass(frozen=True)
class Params:
    eos: EOS
    G: float = -1.0
    kappa: float = 0.0            # surface-tension parameter of Eq. 19
    sigma_force: float = 0.0      # the constant sigma of Eq. 8 (not the surface tension)
    rates: Rates = field(default_factory=Rates)
    walls_y: bool = False         # False: periodic in y; True: no-slip walls below y=0 and above y=ny-1
    # open_bc: no-slip wall below y = 0 and open boundaries (zero-gradient: the missing
    # neighbour takes the value of the boundary site) above y = ny-1 and beyond x = 0,
    # x = nx-1, the droplet-splash geometry of Sec. V.C (the paper does not name its open
    # boundary condition)
    open_bc: bool = False
    # nu(rho) of Sec. V.C: (rho_1, s_v used where rho < rho_1); rates.s_v applies where
    # rho >= rho_1. None: one s_v everywhere.
    visc_switch: tuple = None


# --------------------------------------------------------------------------------------
# a1 .. a9, one function per row
# --------------------------------------------------------------------------------------

def density(f):
    """rho = sum_alpha f_alpha (Eq. 6)."""
    return f.sum(axis=0)


def neighbour(field2d, ex: int, ey: int, walls_y: bool, open_bc: bool = False):
    """field(x + ex, y + ey): periodic in x; periodic in y, or with the value of the
    adjacent fluid row copied into the wall rows y = -1 and y = ny. With open_bc the value
    of the nearest lattice site is used outside the lattice in x and y (zero gradient at
    the open boundaries; the copied wall row below y = 0)."""
    ny, nx = field2d.shape
    if open_bc:
        cols = np.clip(np.arange(nx) + ex, 0, nx - 1)
        rows = np.clip(np.arange(ny) + ey, 0, ny - 1)
        return field2d[rows][:, cols]
    out = np.roll(field2d, shift=-ex, axis=1)
    if not walls_y:
        return np.roll(out, shift=-ey, axis=0)
    rows = np.clip(np.arange(ny) + ey, 0, ny - 1)
    return out[rows, :]


def neighbour_psi(psi, walls_y: bool, open_bc: bool = False):
    """[psi(x + e_alpha) for alpha = 0..8]."""
    return [neighbour(psi, int(EX[a]), int(EY[a]), walls_y, open_bc) for a in range(9)]


def viscosity_rate(rho, p):
    """s_v at every site: rates.s_v, or with nu(rho) (Sec. V.C) the vapour rate where
    rho < rho_1."""
    if p.visc_switch is None:
        return np.full_like(rho, p.rates.s_v)
    rho1, s_v_vapour = p.visc_switch
    return np.where(rho >= rho1, p.rates.s_v, s_v_vapour)


def interaction_force(psi, psi_nb, G: float):
    """F = -G psi(x) sum_{alpha=1..8} w(|e_alpha|^2) psi(x + e_alpha) e_alpha (Eq. 7)."""
    sx = sum(W_INT[a] * psi_nb[a] * EX[a] for a in range(1, 9))
    sy = sum(W_INT[a] * psi_nb[a] * EY[a] for a in range(1, 9))
    return -G * psi * sx, -G * psi * sy


def q_tensor(psi, psi_nb, G: float, kappa: float):
    """Q = kappa (G/2) psi(x) sum_{alpha=1..8} w [psi(x + e_alpha) - psi(x)] e_alpha e_alpha (Eq. 19).
    Returns (Q_xx, Q_yy, Q_xy)."""
    pref = kappa * G / 2.0 * psi
    dxx = sum(W_INT[a] * (psi_nb[a] - psi) * EX[a] * EX[a] for a in range(1, 9))
    dyy = sum(W_INT[a] * (psi_nb[a] - psi) * EY[a] * EY[a] for a in range(1, 9))
    dxy = sum(W_INT[a] * (psi_nb[a] - psi) * EX[a] * EY[a] for a in range(1, 9))
    return pref * dxx, pref * dyy, pref * dxy


def velocity(f, rho, Fx, Fy):
    """rho v = sum_alpha e_alpha f_alpha + F/2 (Eq. 6, delta_t = 1)."""
    jx = sum(EX[a] * f[a] for a in range(9))
    jy = sum(EY[a] * f[a] for a in range(9))
    return (jx + 0.5 * Fx) / rho, (jy + 0.5 * Fy) / rho


def moments(f):
    """m = M f."""
    return np.tensordot(M, f, axes=(1, 0))


def equilibrium_moments(rho, vx, vy):
    """m_eq of Eq. 3."""
    v2 = vx * vx + vy * vy
    return np.stack([
        rho,
        rho * (-2.0 + 3.0 * v2),
        rho * (1.0 - 3.0 * v2),
        rho * vx,
        -rho * vx,
        rho * vy,
        -rho * vy,
        rho * (vx * vx - vy * vy),
        rho * vx * vy,
    ])


def forcing_moments(vx, vy, Fx, Fy, psi, sigma_force: float, s_e: float):
    """S of Eq. 5, with S_1 replaced by Eq. 8 when sigma_force != 0:
    S_1 = 6 (v_x F_x + v_y F_y) + 12 sigma |F|^2 / (psi^2 (tau_e - 0.5)),  S_2 = -S_1."""
    s1 = 6.0 * (vx * Fx + vy * Fy)
    if sigma_force != 0.0:
        tau_e = 1.0 / s_e
        s1 = s1 + 12.0 * sigma_force * (Fx * Fx + Fy * Fy) / (psi * psi * (tau_e - 0.5))
    zero = np.zeros_like(vx)
    return np.stack([
        zero,
        s1,
        -s1,
        Fx,
        -Fx,
        Fy,
        -Fy,
        2.0 * (vx * Fx - vy * Fy),
        vx * Fy + vy * Fx,
    ])


def source_moments(Qxx, Qyy, Qxy, rates: Rates, s_v=None):
    """C of Eq. 18 (its discrete-lattice correction is already included, Sec. IV); s_v
    may be a per-site array (nu(rho))."""
    zero = np.zeros_like(Qxx)
    s_v = rates.s_v if s_v is None else s_v
    tr = Qxx + Qyy
    return np.stack([
        zero,
        1.5 * rates.s_e * tr,
        -1.5 * rates.s_zeta * tr,
        zero,
        zero,
        zero,
        zero,
        -s_v * (Qxx - Qyy),
        -s_v * Qxy,
    ])


def collide(m, meq, S, C, rates: Rates, s_v=None):
    """m* = m - Lambda (m - m_eq) + (I - Lambda/2) S + C (Eq. 17, delta_t = 1); s_v may
    be a per-site array (nu(rho)), the other rates are constants."""
    s = rates.diagonal()[:, None, None] * np.ones_like(m[:1])
    if s_v is not None:
        s[7] = s_v
        s[8] = s_v
    return m - s * (m - meq) + (1.0 - 0.5 * s) * S + C


def stream(fstar, walls_y: bool, open_bc: bool = False):
    """f_alpha(x + e_alpha, t + 1) = f*_alpha(x, t) (Eq. 4), written as a pull.

    With walls in y (half-way bounce-back): a population that would enter the
    lattice from a wall row is replaced by the opposite population that left the
    same site toward that wall, f_alpha(x, t + 1) = f*_opp(alpha)(x, t).
    With open_bc: bounce-back from below y = 0; a population that would enter through
    an open boundary (above y = ny-1, beyond x = 0 or x = nx-1) is pulled from the
    nearest lattice site instead (zero gradient)."""
    ny, nx = fstar.shape[1], fstar.shape[2]
    if open_bc:
        out = np.empty_like(fstar)
        ys, xs = np.mgrid[0:ny, 0:nx]
        for a in range(9):
            ex, ey = int(EX[a]), int(EY[a])
            sy, sx = ys - ey, np.clip(xs - ex, 0, nx - 1)
            wall = sy < 0
            sy = np.clip(sy, 0, ny - 1)
            out[a] = np.where(wall, fstar[OPPOSITE[a]], fstar[a][sy, sx])
        return out
    out = np.empty_like(fstar)
    for a in range(9):
        ex, ey = int(EX[a]), int(EY[a])
        moved = np.roll(fstar[a], shift=ex, axis=1)          # moved[y, x] = f*[y, x - ex]
        if not walls_y:
            out[a] = np.roll(moved, shift=ey, axis=0)        # out[y, x] = f*[y - ey, x - ex]
            continue
        if ey == 0:
            out[a] = moved
        elif ey == 1:
            out[a, 1:, :] = moved[:-1, :]
            out[a, 0, :] = fstar[OPPOSITE[a], 0, :]
        else:  # ey == -1
            out[a, :-1, :] = moved[1:, :]
            out[a, ny - 1, :] = fstar[OPPOSITE[a], ny - 1, :]
    return out


# --------------------------------------------------------------------------------------
# the whole update
# --------------------------------------------------------------------------------------

def step(f, p: Params):
    """One time step f(t) -> f(t + 1): rows a1 .. a9 in order."""
    rho = density(f)                                               # a1
    psi = psi_of_rho(rho, p.eos, p.G)
    psi_nb = neighbour_psi(psi, p.walls_y, p.open_bc)
    Fx, Fy = interaction_force(psi, psi_nb, p.G)                   # a2
    Qxx, Qyy, Qxy = q_tensor(psi, psi_nb, p.G, p.kappa)            # a3
    vx, vy = velocity(f, rho, Fx, Fy)                              # a4
    m = moments(f)                                                 # a5
    meq = equilibrium_moments(rho, vx, vy)
    S = forcing_moments(vx, vy, Fx, Fy, psi, p.sigma_force, p.rates.s_e)   # a6
    s_v = viscosity_rate(rho, p)
    C = source_moments(Qxx, Qyy, Qxy, p.rates, s_v)                # a7
    mstar = collide(m, meq, S, C, p.rates, s_v)                    # a8
    fstar = np.tensordot(M_INV, mstar, axes=(1, 0))
    return stream(fstar, p.walls_y, p.open_bc)                     # a9


def run(f, p: Params, n: int):
    for _ in range(n):
        f = step(f, p)
    return f


def equilibrium(rho, ux, uy):
    """f = M^-1 m_eq(rho, u): the equilibrium populations used as the initial state."""
    return np.tensordot(M_INV, equilibrium_moments(rho, ux, uy), axes=(1, 0))


def macroscopic(f, p: Params):
    """(rho, ux, uy) with the half-force velocity of Eq. 6."""
    rho = density(f)
    psi = psi_of_rho(rho, p.eos, p.G)
    Fx, Fy = interaction_force(psi, neighbour_psi(psi, p.walls_y, p.open_bc), p.G)
    ux, uy = velocity(f, rho, Fx, Fy)
    return rho, ux, uy


def pressure(rho, p: Params):
    """Bulk pressure rho c_s^2 + (G/2) psi^2 (the isotropic part of Eq. 20)."""
    psi = psi_of_rho(rho, p.eos, p.G)
    return rho / 3.0 + 0.5 * p.G * psi * psi
