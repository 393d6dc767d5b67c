"""Host side of the droplet-splash workload (Sec. V.C), on the CPU: the initial state of
`inputs.splash_state` (film, droplet and impact velocity where the paper puts them) and the
spread-radius reading of `splash.spread_radius` (the row 0.1 D above the film, the largest
distance of liquid from the impact axis), against fields whose answers are known."""
import numpy as np
import pytest

from paper_1306_6445_gb300 import inputs as I
from paper_1306_6445_gb300 import splash


def test_splash_state_geometry():
    nx, ny, film, R, gap, U, rl, rv = 600, 225, 25.0, 50.0, 2.0, 0.125, 100.0, 1.0
    rho, ux, uy = I.splash_state(nx, ny, film, R, gap, U, rl, rv)
    assert rho.shape == ux.shape == uy.shape == (ny, nx)
    yc = int(film + R + gap)
    # liquid in the film and at the droplet centre, vapour far from both
    assert rho[5, 10] == pytest.approx(rl, rel=1e-6)
    assert rho[yc, nx // 2] == pytest.approx(rl, rel=1e-6)
    assert rho[ny - 5, 10] == pytest.approx(rv, rel=1e-6)
    # the droplet moves down at U, the film and the vapour are at rest
    assert uy[yc, nx // 2] == pytest.approx(-U, rel=1e-6)
    assert uy[5, 10] == pytest.approx(0.0, abs=1e-12) and np.all(ux == 0)
    # the droplet is symmetric about the impact axis x = nx/2
    assert np.allclose(rho[:, nx // 2 - 40], rho[:, nx // 2 + 40])
    # the film's interface lies at y = film (density midpoint between rows film-1 and film)
    col = rho[:, 10]
    assert col[int(film) - 1] > 0.5 * (rl + rv) > col[int(film)]
    # the gap between droplet and film holds vapour-side densities at the axis
    y_gap = int(film + gap / 2)
    assert rho[y_gap, nx // 2] < rho[yc, nx // 2]


def test_splash_state_overlapping_start():
    # a negative gap starts the droplet inside the film (the start of a splash run): the
    # droplet and the film are one liquid body on the axis, with no vapour between them
    nx, ny, film, R, U, rl, rv = 600, 225, 25.0, 50.0, 0.125, 100.0, 1.0
    rho, _, uy = I.splash_state(nx, ny, film, R, -5.0, U, rl, rv)
    axis = rho[:, nx // 2]
    assert np.all(axis[: int(film + 2 * R - 5) - 2] > 0.5 * (rl + rv))
    assert uy[int(film + R - 5), nx // 2] == pytest.approx(-U, rel=1e-6)


def test_steps_to_counts_from_the_start_time():
    # t* = t0 + U t / D with t0 = 0.05: t* = 0.25 is 160 steps after the start at D = 100
    assert splash.T0 == 0.05
    assert splash.steps_to(0.25, 100.0, 0.125) == 160
    assert splash.steps_to(splash.T0, 100.0, 0.125) == 0


def test_spread_radius_reads_the_film_connected_liquid_above_the_film():
    nx, ny, film, D, rl, rv = 200, 80, 10.0, 40.0, 100.0, 1.0
    mid = 0.5 * (rl + rv)
    rho = np.full((ny, nx), rv)
    rho[: int(film)] = rl                       # the film, rows 0..9
    row = int(film + 0.1 * D)                   # row 14
    rho[int(film):row + 1, 85:121] = rl         # a liquid column standing on the film
    # liquid from x = 85 to 120 with vapour beyond: rho crosses mid halfway to the next
    # site, at 84.5 and 120.5, so the farther edge is 20.5 from the axis x = 100
    assert splash.spread_radius(rho, film, D, rl, rv) == pytest.approx(20.5 / D)
    # a partly filled site beyond the edge moves the edge by the linear crossing of mid
    rho[row, 121] = rv + 0.5 * (mid - rv)       # a quarter of the way from rv to rl
    # crossing between x = 120 (rl) and 121: 120 + (rl - mid) / (rl - rho[121])
    edge = 120 + (rl - mid) / (rl - rho[row, 121])
    assert splash.spread_radius(rho, film, D, rl, rv) == pytest.approx((edge - 100) / D)
    # a detached drop on the row, farther out, does not count (no liquid path to the film)
    rho[row, 185] = rl
    assert splash.spread_radius(rho, film, D, rl, rv) == pytest.approx((edge - 100) / D)
    # liquid connected to the film only through a diagonal does not count (4-neighbours)
    rho2 = np.full((ny, nx), rv)
    rho2[: int(film)] = rl
    rho2[row, 150] = rl
    rho2[row - 1, 151] = rl
    for y in range(int(film), row - 1):
        rho2[y, 151] = rl
    assert splash.spread_radius(rho2, film, D, rl, rv) == pytest.approx(0.0)
