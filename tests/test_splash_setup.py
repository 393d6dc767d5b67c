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


def test_spread_radius_reads_the_row_above_the_film():
    nx, ny, film, D, rl, rv = 200, 80, 10.0, 40.0, 100.0, 1.0
    rho = np.full((ny, nx), rv)
    row = int(film + 0.1 * D)          # row 14
    rho[row, 100 - 30:100 + 21] = rl   # liquid from x = 70 to 120: farthest |x - 100| = 30
    assert splash.spread_radius(rho, film, D, rl, rv) == pytest.approx(30 / D)
    # liquid elsewhere (other rows) does not count
    rho2 = np.full((ny, nx), rv)
    rho2[row + 1, 0:nx] = rl
    rho2[row - 1, 0:nx] = rl
    assert splash.spread_radius(rho2, film, D, rl, rv) == 0.0
    # a detached drop on the row farther out counts (secondary droplets do)
    rho[row, 185] = rl
    assert splash.spread_radius(rho, film, D, rl, rv) == pytest.approx(85 / D)
