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
