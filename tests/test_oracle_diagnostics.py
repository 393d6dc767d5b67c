"""Pins of the oracle's measurement definitions (CPU): the Laplace reading of a sharp
(step) droplet, where every mask mean, the mass radius and the pressure jump follow in
closed form from the EOS, and the interface height's edge cases (NaN where no liquid row
is followed by a vapour row)."""
import numpy as np
import pytest

from oracle import diagnostics as D
from oracle import eos as E
from oracle import lattice as L


def test_laplace_of_a_step_droplet_is_the_closed_form():
    eos = E.cs_eos(0.8)
    p = L.Params(eos=eos, G=-1.0, kappa=0.0, rates=L.Rates.from_viscosity(0.1))
    nx, ny, R = 121, 101, 22.5
    rho_l, rho_v = 0.30, 0.02
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    inside = np.hypot(x - (nx - 1) / 2, y - (ny - 1) / 2) < R
    rho = np.where(inside, rho_l, rho_v)
    d = D.laplace(rho, p)
    # pressure of a uniform phase: rho/3 + (G/2) psi^2 = p_EOS for the EOS-based potential
    p_l = float(E.p_eos(rho_l, eos, -1.0))
    p_v = float(E.p_eos(rho_v, eos, -1.0))
    assert d["rho_in"] == pytest.approx(rho_l, rel=1e-14)
    assert d["rho_out"] == pytest.approx(rho_v, rel=1e-14)
    assert d["p_in"] == pytest.approx(p_l, rel=1e-12)
    assert d["p_out"] == pytest.approx(p_v, rel=1e-12)
    # mass radius of a step field: sqrt(sites inside / pi), close to the drawn radius
    r_mass = np.sqrt(inside.sum() / np.pi)
    assert d["R"] == pytest.approx(r_mass, rel=1e-12)
    assert abs(r_mass - R) < 0.1
    assert d["theta"] == pytest.approx((p_l - p_v) * r_mass, rel=1e-11)


def test_interface_height_edge_cases_are_nan():
    # the first row is already vapour: no liquid below the interface
    assert np.isnan(D.interface_height(np.array([0.1, 0.2, 0.3]), 0.5))
    # no row drops below the threshold: no interface
    assert np.isnan(D.interface_height(np.array([0.9, 0.8, 0.7]), 0.5))
    # the lowest crossing counts, later ones are ignored
    col = np.array([1.0, 0.0, 1.0, 0.0])
    assert D.interface_height(col, 0.5) == pytest.approx(0.5)


def test_interface_height_of_a_tanh_layer_is_the_layer_height():
    # a tanh profile crosses the mean density at its centre h. Linear interpolation between
    # the bracketing rows is exact when h sits on a row or midway between two (the profile
    # is odd about h), and off by the profile's curvature otherwise: under 0.01 rows for a
    # width of 4 rows
    y = np.arange(32, dtype=float)
    mid = 0.5 * (0.3 + 0.02)
    for h, tol in ((10.0, 1e-12), (10.5, 1e-12), (10.25, 1e-2), (10.9, 1e-2)):
        col = mid - 0.5 * (0.3 - 0.02) * np.tanh(2.0 * (y - h) / 4.0)
        assert D.interface_height(col, mid) == pytest.approx(h, abs=tol)


# ---- laplace_fit: the Fig. 3 reading (Sec. V.A), dp = theta / R + c over several radii ----

RADII = np.array([20.0, 25.0, 30.0, 35.0, 40.0])   # the radii of the paper's Laplace test


def test_laplace_fit_recovers_an_exact_line():
    # theta and c of different sizes and signs, so that a swapped column, a dropped
    # intercept or a sign slip cannot reproduce both
    theta, c = 0.8160, -3.0e-4          # Table 3's surface tension at 1 - kappa = 0.5
    dps = theta / RADII + c
    got_t, got_c = D.laplace_fit(dps, RADII)
    assert got_t == pytest.approx(theta, rel=1e-12)
    assert got_c == pytest.approx(c, rel=1e-9)


def test_laplace_fit_through_two_points_is_the_secant():
    # with two radii the least-squares line passes through both points
    r = np.array([20.0, 40.0])
    dps = np.array([0.05, 0.02])
    t, c = D.laplace_fit(dps, r)
    slope = (dps[0] - dps[1]) / (1.0 / r[0] - 1.0 / r[1])
    assert t == pytest.approx(slope, rel=1e-13)
    assert c == pytest.approx(dps[1] - slope / r[1], rel=1e-12)
    assert t == pytest.approx(1.2, rel=1e-12) and c == pytest.approx(-0.01, rel=1e-10)


def test_laplace_fit_of_noisy_data_is_the_textbook_regression():
    # simple linear regression of y on x = 1/R: slope = S_xy / S_xx and intercept
    # = mean(y) - slope mean(x); the residuals are orthogonal to both columns
    rng = np.random.default_rng(1306)
    dps = 9.449 / RADII + rng.normal(0.0, 2e-3, RADII.size)
    t, c = D.laplace_fit(dps, RADII)
    x = 1.0 / RADII
    sxy = np.sum((x - x.mean()) * (dps - dps.mean()))
    sxx = np.sum((x - x.mean()) ** 2)
    assert t == pytest.approx(sxy / sxx, rel=1e-10)
    assert c == pytest.approx(dps.mean() - (sxy / sxx) * x.mean(), abs=1e-12)
    res = dps - (t * x + c)
    assert abs(np.sum(res)) < 1e-13 and abs(np.sum(res * x)) < 1e-14


def test_laplace_fit_of_step_droplets_has_no_slope():
    # sharp (step) droplets of the oracle's Laplace reading: the pressure jump is the
    # bulk difference p_EOS(rho_l) - p_EOS(rho_v) at every radius, so the fit returns a
    # zero surface tension and that difference as its intercept
    eos = E.cs_eos(0.8)
    p = L.Params(eos=eos, G=-1.0, kappa=0.0, rates=L.Rates.from_viscosity(0.1))
    rho_l, rho_v = 0.30, 0.02
    n = 160
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - (n - 1) / 2, y - (n - 1) / 2)
    dps, radii = [], []
    for R in RADII:
        d = D.laplace(np.where(r < R, rho_l, rho_v), p)
        dps.append(d["dp"])
        radii.append(d["R"])
    t, c = D.laplace_fit(dps, radii)
    jump = float(E.p_eos(rho_l, eos, -1.0) - E.p_eos(rho_v, eos, -1.0))
    assert abs(t) < 1e-12 * abs(jump) * 40
    assert c == pytest.approx(jump, rel=1e-12)


def test_zero_crossings_of_a_rippled_damped_cosine():
    """The crossing finder of the capillary-wave test: a damped cosine sampled every 500
    steps with a small fast ripple gives its zero crossings (pi/2 + k pi)/omega to within a
    few steps, each sign change counted once."""
    from _util import zero_crossings
    omega = 2 * np.pi / 110000.0
    ts = np.arange(0, 130001, 500, dtype=float)
    ys = 10.0 * np.exp(-7e-6 * ts) * np.cos(omega * ts) + 0.05 * np.sin(2 * np.pi * ts / 3500.0)
    z = zero_crossings(ts, ys)
    exact = [(np.pi / 2 + k * np.pi) / omega for k in range(2)]
    assert len(z) == 2
    assert np.allclose(z, exact, atol=100.0)
    assert np.pi / (z[1] - z[0]) == pytest.approx(omega, rel=2e-3)
