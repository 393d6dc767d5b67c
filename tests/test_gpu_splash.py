"""Droplet splashing on a thin liquid film (Sec. V.C) on the GPU: 600 x 225, film height 25,
droplet R = 50 moving down at U = 0.125, Eq. 23 fluid (density ratio 100, sigma_F = 0.087),
Re = U D / nu_L = 1000, nu_V / nu_L = 20 switched at rho_1 = 1.49, MRT rates of Sec. V.C,
a no-slip bottom wall and open boundaries elsewhere (LB_BC_OPEN).

The paper does not define its spread radius; it is read here as the largest distance from
the impact axis of liquid (rho above the mean of the phase densities) in the row 0.1 D
above the undisturbed film surface. The droplet starts 2 lattice units above the film."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
T5 = GOLD["table5_splash_spread_radius"]

NX, NY, FILM, R, U = 600, 225, 25.0, 50.0, 0.125
D = 2 * R


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_6445_gb300 import _build

    _build.build()
    from paper_1306_6445_gb300 import lbm as mod

    mod.load_library()
    return mod


def spread_radii(lbm, kappa, tstars, prec="fp32"):
    from paper_1306_6445_gb300 import splash
    nu_l = U * D / 1000.0
    lat = splash.make_lattice(lbm, NX, NY, lbm.EOSParams(kind="piecewise"), -1.0, kappa, 0.087,
                              D, FILM, U, nu_l, 20.0 * nu_l, 1.49, 100.0, 1.0, prec=prec)
    out, done = [], 0
    for ts in tstars:
        n = int(round(ts * D / U))
        lat.step(n - done)
        done = n
        out.append(splash.spread_radius(lat.rho(), FILM, D, 100.0, 1.0))
    lat.close()
    return np.array(out)


def test_spread_radius_follows_table5_and_the_power_law(lbm):
    ts = np.array(T5["t_star"][1:])                 # 0.25, 0.75, 1.0, 1.5
    r0 = spread_radii(lbm, 0.0, ts)
    r1 = spread_radii(lbm, 0.75, ts)
    print("t*", ts, "r/D (1-kappa = 1)", r0, "(1-kappa = 0.25)", r1,
          "Table 5", T5["r_over_D_one_minus_kappa_1"][1:])
    # the power law r/D ~ 1.3 sqrt(t*) (the paper's own values lie within 4 % of it)
    assert np.all(np.abs(r0 / (1.3 * np.sqrt(ts)) - 1) < 0.06)
    # Table 5, 1 - kappa = 1, within 5 % (open-boundary type, start gap and the radius
    # measure are readings)
    assert np.all(np.abs(r0 / np.array(T5["r_over_D_one_minus_kappa_1"][1:]) - 1) < 0.05)
    # the surface tension barely changes the spread radius (Table 5's conclusion)
    assert np.all(np.abs(r1 / r0 - 1) < 0.03)


def test_fp32_and_fp64_spread_radii_agree(lbm):
    ts = np.array([0.25, 1.0])
    a = spread_radii(lbm, 0.0, ts, "fp32")
    b = spread_radii(lbm, 0.0, ts, "fp64")
    assert np.all(np.abs(a - b) <= 2.0 / D)         # within two lattice units
