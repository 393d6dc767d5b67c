"""Pins of the oracle's thermodynamic tools: closed forms from the literature,
finite differences, and the coexistence densities the paper prints. CPU only."""
import json
import os

import numpy as np
import pytest

from oracle import diagnostics as D
from oracle import eos as E

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_cs_critical_point_matches_known_constant():
    """Carnahan-Starling: b R T_c / a = 0.3773 and b rho_c = 0.5218 (textbook values)."""
    for a, b, R in [(1.0, 4.0, 1.0), (0.5, 2.0, 1.0), (2.0, 4.0, 0.5)]:
        Tc, rc = E.cs_critical(a, b, R)
        assert b * R * Tc / a == pytest.approx(0.37731, abs=2e-5)
        assert b * rc == pytest.approx(0.52178, abs=2e-5)
        eos = E.EOS(kind="cs", a=a, b=b, R=R, T=Tc)
        h = 1e-4 * rc
        d1 = (E.p_eos(rc + h, eos, -1) - E.p_eos(rc - h, eos, -1)) / (2 * h)
        d2 = (E.p_eos(rc + h, eos, -1) - 2 * E.p_eos(rc, eos, -1) + E.p_eos(rc - h, eos, -1)) / h**2
        scale = float(E.p_eos(rc, eos, -1)) / rc
        assert abs(d1) < 1e-7 * scale and abs(d2) < 1e-3 * scale / rc


@pytest.mark.parametrize("eos,G", [(E.cs_eos(0.8), -1.0), (E.EOS(kind="exp"), -40.0),
                                   (E.colosqui_eos(), -1.0)])
def test_dp_drho_matches_finite_difference(eos, G):
    rhos = {"cs": [0.01, 0.1, 0.3], "exp": [50.0, 200.0, 600.0], "piecewise": [0.5, 20.0, 98.0]}
    for r in rhos[eos.kind]:
        h = 1e-6 * r
        fd = (E.p_eos(r + h, eos, G) - E.p_eos(r - h, eos, G)) / (2 * h)
        assert float(E.dp_drho(r, eos, G)) == pytest.approx(float(fd), rel=1e-6, abs=1e-12)


def _mu_cs(rho, eos):
    """Chemical potential of CS + mean field, known closed form:
    mu = R T [ln rho + (8 eta - 9 eta^2 + 3 eta^3)/(1 - eta)^3] - 2 a rho."""
    eta = eos.b * rho / 4
    return eos.R * eos.T * (np.log(rho) + (8 * eta - 9 * eta**2 + 3 * eta**3) / (1 - eta) ** 3) \
        - 2 * eos.a * rho


def _mu_exp(rho, eos, G):
    """mu = int dp / rho for p = rho/3 + (G/2) psi0^2 exp(-2 rho0/rho), in closed form:
    (1/3) ln rho + (G/2) psi0^2 exp(-2 rho0/rho) (1/rho + 1/(2 rho0))."""
    return np.log(rho) / 3 + 0.5 * G * eos.psi0**2 * np.exp(-2 * eos.rho0 / rho) * (
        1 / rho + 1 / (2 * eos.rho0))


@pytest.mark.parametrize("t", [0.7, 0.8, 0.9])
def test_cs_maxwell_equal_pressure_and_chemical_potential(t):
    eos = E.cs_eos(t)
    rv, rl, pb = E.maxwell(eos, -1.0)
    assert float(E.p_eos(rv, eos, -1)) == pytest.approx(pb, rel=1e-10)
    assert float(E.p_eos(rl, eos, -1)) == pytest.approx(pb, rel=1e-10)
    assert _mu_cs(rv, eos) == pytest.approx(_mu_cs(rl, eos), rel=1e-9)


def test_exp_maxwell_matches_paper_and_closed_form_mu():
    g = GOLD["maxwell_exp_psi"]
    eos = E.EOS(kind="exp", psi0=g["psi0"], rho0=g["rho0"])
    rv, rl, pb = E.maxwell(eos, g["G"])
    assert rl == pytest.approx(g["rho_l"], rel=3e-3)     # paper: "rho_L ~ 514"
    assert rv == pytest.approx(g["rho_v"], rel=3e-3)     # paper: "rho_V ~ 79.5"
    assert _mu_exp(rv, eos, g["G"]) == pytest.approx(_mu_exp(rl, eos, g["G"]), rel=1e-9)


def test_colosqui_maxwell_matches_paper():
    g = GOLD["colosqui_coexistence"]
    rv, rl, pb = E.maxwell(E.colosqui_eos(), g["G"])
    assert rl == pytest.approx(g["rho_l"], rel=1e-3)
    assert rv == pytest.approx(g["rho_v"], rel=5e-3)


def test_eq16_eps0_equals_maxwell_for_exponential_potential():
    """For psi = psi0 exp(-rho0/rho), psi'/psi = rho0/rho^2, so Eq. 16 with eps = 0 is
    the Maxwell rule (Sec. II: thermodynamically consistent with Eq. 5)."""
    eos = E.EOS(kind="exp")
    a = E.maxwell(eos, -40.0)
    b = E.mechanical_stability(eos, -40.0, 0.0)
    assert b[0] == pytest.approx(a[0], rel=1e-8) and b[1] == pytest.approx(a[1], rel=1e-8)


def test_eq16_gives_lower_vapour_density_than_maxwell_for_cs():
    """Sec. II: with the EOS-based psi and Eq. 5 the LB coexistence departs from Maxwell."""
    eos = E.cs_eos(0.8)
    mv, ml, _ = E.maxwell(eos, -1.0)
    sv, sl, _ = E.mechanical_stability(eos, -1.0, 0.0)
    assert sv < 0.5 * mv and abs(sl - ml) / ml < 0.02


def test_psi_domain_error():
    eos = E.cs_eos(0.8)
    with pytest.raises(E.DomainError):
        E.psi_of_rho(np.array([0.1, 0.6]), eos, -1.0)
    with pytest.raises(E.DomainError):
        E.psi_of_rho(np.array([-0.01]), eos, -1.0)


def test_flat_surface_tension_quadrature_near_paper_table2():
    """Continuum flat-interface theta (from Eq. 22) vs the paper's LB value at kappa = 0
    (Table 2, 9.449 at R = 40); the lattice value is a few percent below the continuum."""
    eos = E.EOS(kind="exp")
    th = E.flat_surface_tension(eos, -40.0, 0.0)
    assert th == pytest.approx(GOLD["table2_exp_psi"]["surface_tension"][0], rel=0.03)
    # theta is exactly linear in (1 - kappa) in this continuum form
    assert E.flat_surface_tension(eos, -40.0, 0.5) == pytest.approx(0.5 * th, rel=1e-12)


def test_capillary_dispersion_reproduces_table4_from_table3():
    """With Table 3's theta (1 - kappa = 1, 0.5), omega^2 = theta k^3/(rho_L + rho_V)
    gives Table 4's analytical periods; the printed Eq. 24 without the square cannot."""
    t3, t4 = GOLD["table3_colosqui"], GOLD["table4_capillary"]
    for i in range(2):
        T = D.capillary_period(t3["surface_tension"][i], t4["wavelength"], t4["rho_l"], t4["rho_v"])
        assert T == pytest.approx(t4["analytical_period"][i], rel=0.012)
    # literal (unsquared) reading: omega = theta k^3 / (rho_L + rho_V)
    k = 2 * np.pi / t4["wavelength"]
    T_literal = 2 * np.pi / (t3["surface_tension"][0] * k**3 / (t4["rho_l"] + t4["rho_v"]))
    assert T_literal > 100 * t4["analytical_period"][0]


def test_finite_depth_dispersion_tends_to_deep_limit():
    deep = D.capillary_period(0.01, 256, 0.3, 0.02)
    assert D.capillary_period(0.01, 256, 0.3, 0.02, 1e4, 1e4) == pytest.approx(deep, rel=1e-12)
    assert D.capillary_period(0.01, 256, 0.3, 0.02, 20, 20) > deep


def test_interface_height_linear_interpolation():
    col = np.array([1.0, 1.0, 0.8, 0.4, 0.0, 0.0])
    assert D.interface_height(col, 0.5) == pytest.approx(2.75)


def test_splash_weber_numbers_follow_eq22_and_table3():
    """Sec. V.C's Weber numbers against the rest of the paper: their ratio is the (1 - kappa)
    scaling of Eq. 22 between kappa = 0 and 0.95, and rho_l U^2 D / We(kappa = 0) is Table 3's
    surface tension of the same fluid at 1 - kappa = 1 (rho_l of Sec. V.A). This fixes the
    reading We = rho_l U^2 D / theta with D = 2R that the splash set-up uses."""
    w, t3, co = GOLD["splash_weber"], GOLD["table3_colosqui"], GOLD["colosqui_coexistence"]
    k0, k1 = w["kappa"]
    assert w["We"][1] / w["We"][0] == pytest.approx((1 - k0) / (1 - k1), rel=0.01)
    theta0 = co["rho_l"] * w["U"] ** 2 * w["D"] / w["We"][0]
    assert theta0 == pytest.approx(t3["surface_tension"][0], rel=0.02)
