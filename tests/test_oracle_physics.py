"""Physics pins of the oracle's lattice update against the paper's theory and
printed numbers: coexistence densities of flat interfaces (Eq. 16 / Maxwell),
their independence of kappa (Eq. 22), the improved forcing (Eq. 8, Table 3) and
the Laplace law with theta proportional to (1 - kappa) (Table 2). CPU only;
each run is small enough to converge in a few seconds."""
import json
import os

import numpy as np
import pytest

from oracle import diagnostics as D
from oracle import eos as E
from oracle import lattice as L
from paper_1306_6445_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def slab(eos, G, rho_l, rho_v, ny, kappa=0.0, sigma=0.0, steps=3000, width=4.0):
    rho = I.layer_density(4, ny, ny / 2, rho_l, rho_v, width=width, y_offset=ny / 4,
                          two_sided=True)
    f = L.equilibrium(rho, 0 * rho, 0 * rho)
    p = L.Params(eos=eos, G=G, kappa=kappa, sigma_force=sigma, rates=L.Rates.from_viscosity(0.1))
    f = L.run(f, p, steps)
    return D.slab_densities(L.density(f))


def droplet(eos, G, rho_l, rho_v, n, R, kappa, steps=2500):
    rho = I.droplet_density(n, n, R, rho_l, rho_v)
    f = L.equilibrium(rho, 0 * rho, 0 * rho)
    p = L.Params(eos=eos, G=G, kappa=kappa, rates=L.Rates.from_viscosity(0.1))
    f = L.run(f, p, steps)
    return D.laplace(L.density(f), p)


def test_flat_interface_exp_psi_reaches_maxwell():
    """Sec. II: psi0 exp(-rho0/rho) with Eq. 5 is thermodynamically consistent."""
    eos = E.EOS(kind="exp")
    mv, ml, _ = E.maxwell(eos, -40.0)
    rv, rl = slab(eos, -40.0, ml, mv, 64)
    assert rv == pytest.approx(mv, rel=5e-3)
    assert rl == pytest.approx(ml, rel=2e-3)


def test_flat_interface_cs_follows_eq16():
    """CS with Eq. 5: the lattice coexistence is the eps = 0 solution of Eq. 16."""
    eos = E.cs_eos(0.8)
    pv, pl, _ = E.mechanical_stability(eos, -1.0, 0.0)
    rv, rl = slab(eos, -1.0, pl, pv, 64)
    assert rv == pytest.approx(pv, rel=1e-3)
    assert rl == pytest.approx(pl, rel=1e-4)


def test_flat_interface_densities_do_not_move_with_kappa():
    """Eq. 22: P_nn = p0 + (G/4) psi psi'' for every kappa, so the coexistence densities
    stay put (the paper reports a 0.8% change of the density ratio, Sec. V.A)."""
    eos = E.cs_eos(0.8)
    pv, pl, _ = E.mechanical_stability(eos, -1.0, 0.0)
    base = slab(eos, -1.0, pl, pv, 64, kappa=0.0)
    for kappa in (0.5, 0.9):
        rv, rl = slab(eos, -1.0, pl, pv, 64, kappa=kappa)
        assert rv == pytest.approx(base[0], rel=0.02)
        assert rl == pytest.approx(base[1], rel=1e-3)


def test_improved_forcing_reaches_paper_densities_for_piecewise_eos():
    """Eq. 8 with sigma = 0.087 and the EOS of Eq. 23 gives rho_L ~ 100, rho_V ~ 1
    (Sec. V.A, Table 3); without the term Eq. 16 (eps = 0) has no solution."""
    g = GOLD["colosqui_coexistence"]
    rv, rl = slab(E.colosqui_eos(), g["G"], g["rho_l"], g["rho_v"], 128,
                  sigma=g["sigma_force"], steps=4000, width=5.0)
    assert rl == pytest.approx(g["rho_l"], rel=2e-3)
    assert rv == pytest.approx(g["rho_v"], rel=0.05)
    with pytest.raises(ValueError):
        E.mechanical_stability(E.colosqui_eos(), g["G"], 0.0)


def test_laplace_theta_scales_with_one_minus_kappa_exp_psi():
    """Table 2: theta(kappa = 0.5) / theta(0) = 4.605 / 9.449; densities unchanged."""
    eos = E.EOS(kind="exp")
    mv, ml, _ = E.maxwell(eos, -40.0)
    d0 = droplet(eos, -40.0, ml, mv, 48, 14.0, 0.0)
    d5 = droplet(eos, -40.0, ml, mv, 48, 14.0, 0.5)
    t2 = GOLD["table2_exp_psi"]["surface_tension"]
    assert d5["theta"] / d0["theta"] == pytest.approx(t2[1] / t2[0], rel=0.02)
    # R = 14 here, R = 40 in the paper: a few percent of finite-size difference
    assert d0["theta"] == pytest.approx(t2[0], rel=0.05)
    # density ratio: the paper sees 0.8% over kappa in [0, 0.99] at R = 40 and ascribes it
    # to higher-order (curvature) terms, which are larger at R = 14
    assert d5["rho_in"] / d5["rho_out"] == pytest.approx(d0["rho_in"] / d0["rho_out"], rel=0.015)
    # Laplace law sign and the mass-derived radius
    assert d0["dp"] > 0 and d0["R"] == pytest.approx(14.0, abs=0.5)


def test_laplace_theta_cs_near_flat_interface_theory():
    """CS, 0.8 Tc, Eq. 5: the droplet's theta is within 10% of the continuum flat-interface
    value of Eq. 22 and halves at kappa = 0.5."""
    eos = E.cs_eos(0.8)
    pv, pl, _ = E.mechanical_stability(eos, -1.0, 0.0)
    d0 = droplet(eos, -1.0, pl, pv, 48, 14.0, 0.0)
    d5 = droplet(eos, -1.0, pl, pv, 48, 14.0, 0.5)
    th = E.flat_surface_tension(eos, -1.0, 0.0)
    assert d0["theta"] == pytest.approx(th, rel=0.10)
    assert d5["theta"] / d0["theta"] == pytest.approx(0.5, abs=0.03)
