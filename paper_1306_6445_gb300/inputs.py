"""Seeded synthetic inputs for the lattice runs.

This module holds only initial-condition geometry and random numbers: density
and velocity fields (a tanh droplet, a flat or cosine-perturbed layer, a shear
wave), random population arrays and random parameter draws for batches. It
contains none of the update's arithmetic (no equilibrium, EOS or collision):
each consumer turns (rho, u) into populations with its own code.

Every generator is deterministic for a given seed. The paper draws no random
numbers; randomness only appears in parity inputs and in the batched sweep.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 1306


def droplet_density(nx: int, ny: int, radius: float, rho_l: float, rho_v: float,
                    width: float = 2.0, center=None) -> np.ndarray:
    """Circular droplet, liquid inside, with a tanh interface of the given width:
    rho(r) = (rho_l + rho_v)/2 - (rho_l - rho_v)/2 tanh(2 (r - R) / width).
    Centre ((nx-1)/2, (ny-1)/2) by default. Shape (ny, nx), float64."""
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.hypot(x - center[0], y - center[1])
    return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (r - radius) / width)


def layer_density(nx: int, ny: int, height: float, rho_l: float, rho_v: float,
                  width: float = 2.0, amplitude: float = 0.0, wavenumber: int = 1,
                  y_offset: float = 0.0, two_sided: bool = False) -> np.ndarray:
    """Liquid layer below the interface y_i(x) = y_offset + height + amplitude cos(2 pi k x / nx).

    two_sided=False: liquid for y < y_i (a film on the bottom wall, vapour above).
    two_sided=True: a liquid slab between y_offset and y_i (two flat interfaces,
    for periodic lattices). Shape (ny, nx), float64."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    yi = y_offset + height + amplitude * np.cos(2.0 * np.pi * wavenumber * x / nx)
    upper = np.tanh(2.0 * (y - yi) / width)
    if not two_sided:
        return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * upper
    lower = np.tanh(2.0 * (y_offset - y) / width)
    # liquid where both tanh terms are negative (between the two interfaces)
    frac = 0.25 * (1.0 - upper) * (1.0 - lower)
    return rho_v + (rho_l - rho_v) * frac


def shear_wave(nx: int, ny: int, amplitude: float, rho: float = 1.0):
    """rho uniform, u_x = U sin(2 pi y / ny), u_y = 0. Returns (rho, ux, uy)."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    ux = amplitude * np.sin(2.0 * np.pi * y / ny)
    return np.full((ny, nx), rho), ux, np.zeros((ny, nx))


def smooth_random_density(rng: np.random.Generator, nx: int, ny: int, rho_lo: float,
                          rho_hi: float, modes: int = 3) -> np.ndarray:
    """A smooth periodic density field in [rho_lo, rho_hi] built from a few random
    Fourier modes (so that neighbour differences are interface-like, not noise)."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    acc = np.zeros((ny, nx))
    for _ in range(modes):
        kx, ky = rng.integers(1, 4, size=2)
        ph = rng.uniform(0, 2 * np.pi)
        acc += np.cos(2 * np.pi * (kx * x / nx + ky * y / ny) + ph)
    acc = (acc - acc.min()) / max(acc.max() - acc.min(), 1e-300)
    return rho_lo + (rho_hi - rho_lo) * acc


def random_populations(rng: np.random.Generator, rho: np.ndarray, spread: float = 0.3) -> np.ndarray:
    """Non-equilibrium populations f[alpha, y, x] >= 0 whose sum is rho (up to rounding):
    each site splits rho over the nine directions with random positive fractions
    around 4/9, 1/9, 1/36. The fractions are input noise, not an equilibrium."""
    base = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    noise = rng.uniform(1.0 - spread, 1.0 + spread, size=(9,) + rho.shape)
    frac = base[:, None, None] * noise
    frac /= frac.sum(axis=0, keepdims=True)
    return frac * rho[None, :, :]


def random_velocity(rng: np.random.Generator, shape, umax: float):
    return rng.uniform(-umax, umax, size=shape), rng.uniform(-umax, umax, size=shape)


def batch_draws(n: int = 512, seed: int = DEFAULT_SEED):
    """Random lattice descriptors for a batched Laplace-law sweep: side from
    {64, 96, ..., 512}, radius fraction U[0.15, 0.35], T/Tc U[0.65, 0.95],
    kappa U[0, 0.95], tau_v U[0.6, 1.2]. Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    sides = np.arange(64, 513, 32)
    out = []
    for _ in range(n):
        side = int(rng.choice(sides))
        out.append({
            "side": side,
            "radius": float(rng.uniform(0.15, 0.35) * side),
            "t_over_tc": float(rng.uniform(0.65, 0.95)),
            "kappa": float(rng.uniform(0.0, 0.95)),
            "tau_v": float(rng.uniform(0.6, 1.2)),
        })
    return out


def mlp_init(seed: int = DEFAULT_SEED, n_in: int = 3, hidden: int = 64, n_out: int = 3):
    """Initial parameters of the surrogate network as one float32 vector in the layout
    W1[h][in], b1[h], W2[h][h], b2[h], W3[out][h], b3[out]: weights uniform in
    +-sqrt(6 / (fan_in + fan_out)) (Glorot & Bengio 2010), biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for fi, fo in ((n_in, hidden), (hidden, hidden), (hidden, n_out)):
        a = np.sqrt(6.0 / (fi + fo))
        parts += [rng.uniform(-a, a, fo * fi), np.zeros(fo)]
    return np.concatenate(parts).astype(np.float32)


def mlp_random_data(n: int, seed: int = DEFAULT_SEED):
    """Random training pairs for gradient checks: x = (T/T_c, kappa, tau_v) uniform over the
    sweep's ranges, y = (sigma, rho_l, rho_v) positive and spread over the ranges the
    sweep produces (sigma and rho_v log-uniform). float32, n x 3 each."""
    rng = np.random.default_rng(seed)
    x = np.stack([rng.uniform(0.65, 0.95, n), rng.uniform(0.0, 0.95, n),
                  rng.uniform(0.6, 1.2, n)], axis=1)
    y = np.stack([np.exp(rng.uniform(np.log(2e-5), np.log(1e-2), n)),
                  rng.uniform(0.3, 0.6, n), np.exp(rng.uniform(np.log(1e-3), np.log(0.15), n))],
                 axis=1)
    return x.astype(np.float32), y.astype(np.float32)


def splash_state(nx: int, ny: int, film: float, radius: float, gap: float, speed: float,
                 rho_l: float, rho_v: float, width: float = 2.0):
    """Droplet above a liquid film (Sec. V.C): a film of height `film` on the bottom and a
    droplet of `radius` centred at (nx/2, film + radius + gap) moving down at `speed`;
    tanh interfaces of the given width. Returns (rho, ux, uy) as [ny][nx] arrays."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    xc, yc = 0.5 * nx, film + radius + gap
    f_film = 0.5 * (1.0 - np.tanh(2.0 * (y + 0.5 - film) / width))
    f_drop = 0.5 * (1.0 - np.tanh(2.0 * (np.hypot(x - xc, y - yc) - radius) / width))
    rho = rho_v + (rho_l - rho_v) * np.maximum(f_film, f_drop)
    ux = np.zeros_like(rho)
    uy = -speed * f_drop
    return rho, ux, uy
