"""Physics of the CUDA path against what the paper prints (GPU, FP64 unless stated).

Laplace measurements use the oracle's reading of the method (tests may use the oracle);
every run is converged (the droplets change by < 1e-5 over the last chunks of these
step counts). Tolerances state how far the paper's own numbers can be expected to be
matched given the readings of the paper's silences (relaxation rates other than s_v and
the measurement masks are not given in the paper)."""
import json
import os

import numpy as np
import pytest

from oracle import diagnostics as D
from oracle import eos as OE
from paper_1306_6445_gb300 import inputs as I

from _util import oracle_params

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_6445_gb300 import _build

    _build.build()
    from paper_1306_6445_gb300 import lbm as mod

    mod.load_library()
    return mod


def droplet(lbm, eos, G, n, R, rho_l, rho_v, kappa, sigma, nu, prec, steps):
    rates = lbm.RateParams.from_viscosity(nu)
    lat = lbm.Lattice(n, n, eos, G, kappa=kappa, sigma_force=sigma, rates=rates, prec=prec)
    lat.set_rho_u(I.droplet_density(n, n, R, rho_l, rho_v))
    m0 = lat.reduce()
    lat.step(steps)
    rho = lat.rho()
    m1 = lat.reduce()
    lat.close()
    d = D.laplace(rho, oracle_params(eos, G, kappa, sigma, rates))
    d["mass_drift"] = abs(m1[0] - m0[0]) / m0[0]
    d["umax"] = m1[3]
    print(f"droplet {eos.kind} n={n} R={R} kappa={kappa} sigma={sigma} {prec}: "
          + ", ".join(f"{k}={v:.6g}" for k, v in d.items()))
    return d


def test_table2_exponential_potential_droplets(lbm):
    """Sec. V.A, Table 2 and the text under Fig. 2: 120^2, R = 40, nu = 0.1, psi0 = 4,
    rho0 = 200, G = -40."""
    eos = lbm.EOSParams(kind="exp")
    mv, ml, _ = lbm.lb_maxwell(eos, -40.0)
    t2 = GOLD["table2_exp_psi"]
    fig2 = GOLD["fig2_densities_exp_psi"]
    res = {k: droplet(lbm, eos, -40.0, 120, 40.0, ml, mv, k, 0.0, 0.1, "fp64", 45000)
           for k in (0.0, 0.5, 0.95, 0.99)}
    d0 = res[0.0]
    # coexistence densities at kappa = 0: 517.5 / 80.1, ratio 6.461
    assert d0["rho_in"] == pytest.approx(fig2["rho_l"][0], rel=3e-3)
    assert d0["rho_out"] == pytest.approx(fig2["rho_v"][0], rel=3e-3)
    assert d0["rho_in"] / d0["rho_out"] == pytest.approx(fig2["ratio"][0], rel=3e-3)
    # surface tension at kappa = 0 and 0.5 (Table 2) within 5 %
    assert d0["theta"] == pytest.approx(t2["surface_tension"][0], rel=0.05)
    assert res[0.5]["theta"] == pytest.approx(t2["surface_tension"][1], rel=0.05)
    # theta follows (1 - kappa) (Eq. 22) to within 5 % up to kappa = 0.95
    for k in (0.5, 0.95):
        assert res[k]["theta"] / d0["theta"] == pytest.approx(1 - k, rel=0.05)
    # kappa = 0.95 and 0.99: the surface tension left is a higher-order term. The paper's
    # own values there fall below (1 - kappa) theta(0) by 0.8 % and 0.6 % of theta(0); the
    # printed values are matched to 1.2 % of theta(0) (an absolute tolerance of that size),
    # and theta keeps falling towards zero
    for k, t_paper in zip(t2["kappa"][2:], t2["surface_tension"][2:]):
        assert abs(res[k]["theta"] - t_paper) < 0.012 * t2["surface_tension"][0]
    assert 0 < res[0.99]["theta"] < res[0.95]["theta"] < res[0.5]["theta"]
    # the density ratio moves by less than 1 % (paper: 0.8 % over kappa in [0, 0.99])
    for k in (0.5, 0.95, 0.99):
        r = res[k]["rho_in"] / res[k]["rho_out"]
        assert r == pytest.approx(d0["rho_in"] / d0["rho_out"], rel=0.01)
    for d in res.values():
        assert d["mass_drift"] < 1e-12   # FP64, f*_0 closed by mass conservation


def test_table3_piecewise_eos_droplets(lbm):
    """Sec. V.A, Table 3: EOS of Eq. 23, G = -1, sigma = 0.087 (Eq. 8), R = 40."""
    eos = lbm.EOSParams(kind="piecewise")
    t3 = GOLD["table3_colosqui"]
    for i, omk in enumerate(t3["one_minus_kappa"]):
        d = droplet(lbm, eos, -1.0, 128, 40.0, 100.0, 1.0, 1 - omk, 0.087, 0.1, "fp64", 30000)
        assert d["rho_in"] == pytest.approx(t3["rho_l"][i], rel=1e-3)
        assert d["rho_out"] == pytest.approx(t3["rho_v"][i], rel=0.01)
        if omk >= 0.05:
            tol = 0.01 if omk >= 0.5 else 0.05
            assert d["theta"] == pytest.approx(t3["surface_tension"][i], rel=tol)
        else:
            # 1 - kappa = 0.01: the higher-order residual (see the Table 2 test); within
            # 1.2 % of theta at kappa = 0
            assert abs(d["theta"] - t3["surface_tension"][i]) < 0.012 * t3["surface_tension"][0]
        assert d["mass_drift"] < 1e-12


def test_laplace_law_is_linear_in_inverse_radius(lbm):
    """Sec. V.A, Fig. 3: dp = theta / R over 20 <= R <= 40 (Eq. 23 EOS, 1 - kappa = 1)."""
    eos = lbm.EOSParams(kind="piecewise")
    radii, dps = [], []
    for R in (20.0, 25.0, 30.0, 35.0, 40.0):
        d = droplet(lbm, eos, -1.0, 128, R, 100.0, 1.0, 0.0, 0.087, 0.1, "fp64", 25000)
        radii.append(d["R"])
        dps.append(d["dp"])
    theta, c = D.laplace_fit(dps, radii)
    print("laplace radii", radii, "dp", dps, "theta", theta, "intercept", c)
    pred = theta / np.array(radii) + c
    assert np.max(np.abs(pred - dps)) < 0.01 * max(dps)          # a straight line in 1/R
    # nearly through the origin: the diffuse interface (about five lattice units wide)
    # shifts the line by a few percent of dp at R = 20; the paper claims only linearity
    assert abs(c) < 0.05 * max(dps)
    # the slope of the line is within 7 % of the single-radius value at R = 40, which the
    # paper reports in Table 3 (the small intercept above tilts the fitted slope)
    assert theta == pytest.approx(GOLD["table3_colosqui"]["surface_tension"][0], rel=0.07)


def capillary_period(lbm, one_minus_kappa, steps=18000, every=50):
    L, H = 160, 560
    eos = lbm.EOSParams(kind="piecewise")
    rates = lbm.RateParams.from_viscosity(0.01)
    lat = lbm.Lattice(L, H, eos, -1.0, kappa=1 - one_minus_kappa, sigma_force=0.087,
                      rates=rates, prec="fp64", walls_y=True)
    lat.set_rho_u(I.layer_density(L, H, H / 2, 100.0, 1.0, width=5.0, amplitude=0.125 * L))
    ts, hs = [], []
    while lat.steps_done <= steps:
        hs.append(D.interface_height(lat.rho()[:, 0], 0.5 * (100.0 + 1.0)) - H / 2)
        ts.append(lat.steps_done)
        lat.step(every)
    lat.close()
    ts, hs = np.array(ts, float), np.array(hs)
    z = [ts[i] - hs[i] * (ts[i + 1] - ts[i]) / (hs[i + 1] - hs[i])
         for i in range(len(hs) - 1) if hs[i] * hs[i + 1] < 0]
    return 2.0 * np.mean(np.diff(z)), hs[0]


def test_capillary_wave_periods_follow_dispersion_relation(lbm):
    """Sec. V.B, Table 4: L = 160, H = 3.5 L, h0 = 0.125 L, nu = 0.01, rho_L/rho_V = 100,
    walls in y. The periods agree with the analytical periods (Eq. 24 read with omega^2)
    to within 2.5 % (the paper's own errors: 3.3 %, 0.9 %, 3.5 %), and at 1 - kappa = 0.25
    within 2 % of the paper's numerical period. Runs cover about two periods."""
    t4 = GOLD["table4_capillary"]
    for i, omk in enumerate(t4["one_minus_kappa"]):
        T, h0 = capillary_period(lbm, omk, steps=int(2.3 * t4["analytical_period"][i]))
        print(f"capillary 1-kappa={omk}: period {T:.1f} (analytical {t4['analytical_period'][i]},"
              f" paper {t4['numerical_period'][i]})")
        assert h0 == pytest.approx(0.125 * t4["wavelength"], abs=1.0)
        assert T == pytest.approx(t4["analytical_period"][i], rel=0.025)
        if omk == 0.25:
            assert T == pytest.approx(t4["numerical_period"][i], rel=0.02)


def test_fp32_matches_fp64_on_a_converged_droplet(lbm):
    """FP32 storage and arithmetic against the FP64 path: density ratio and Laplace surface
    tension within 0.5 % on converged droplets (CS at 0.8 T_c, started from the Eq. 16
    coexistence densities, 256^2, R = 50, nu = 0.1, kappa = 0 and 0.6)."""
    eos = lbm.cs_eos(0.8)
    oeos = OE.EOS(kind="cs", T=eos.T)
    pv, pl, _ = OE.mechanical_stability(oeos, -1.0, 0.0)
    for kappa in (0.0, 0.6):
        a = droplet(lbm, eos, -1.0, 256, 50.0, pl, pv, kappa, 0.0, 0.1, "fp64", 40000)
        b = droplet(lbm, eos, -1.0, 256, 50.0, pl, pv, kappa, 0.0, 0.1, "fp32", 40000)
        ra, rb = a["rho_in"] / a["rho_out"], b["rho_in"] / b["rho_out"]
        assert rb == pytest.approx(ra, rel=5e-3)
        assert b["theta"] == pytest.approx(a["theta"], rel=5e-3)
        # FP32 mass drift: a converged (stationary) state repeats the same roundings every
        # step, so the lattice-wide error of ~sqrt(N) ulp per step adds up linearly
        # (~1e-9 per step here); FP64 keeps it below 1e-13
        assert b["mass_drift"] < 2e-4 and a["mass_drift"] < 1e-12
        # spurious currents: no paper value (parity unpinned); FP32 within 10 % of FP64
        assert b["umax"] == pytest.approx(a["umax"], rel=0.1)
