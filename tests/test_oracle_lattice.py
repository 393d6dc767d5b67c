"""Pins of the oracle's lattice update against things other than itself:
textbook D2Q9 formulas, exact invariants, a closed-form decay rate and the
velocity-space brute-force twin. CPU only."""
import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import eos as E
from oracle import lattice as L
from paper_1306_6445_gb300 import inputs as I

W_EQ = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
E_VEC = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]


def textbook_feq(rho, ux, uy):
    """D2Q9 second-order equilibrium, w_a rho (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u^2)."""
    out = np.empty((9,) + np.shape(rho))
    u2 = ux * ux + uy * uy
    for a, (ex, ey) in enumerate(E_VEC):
        eu = ex * ux + ey * uy
        out[a] = W_EQ[a] * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * u2)
    return out


def rates_all(s):
    return L.Rates(s_rho=s, s_e=s, s_zeta=s, s_j=s, s_q=s, s_v=s)


# ---------------------------------------------------------------- M and equilibria

def test_m_rows_orthogonal_with_standard_norms():
    gram = L.M @ L.M.T
    assert np.array_equal(gram, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]).astype(float))
    assert np.allclose(L.M_INV @ L.M, np.eye(9), atol=1e-15)


def test_m_matches_polynomial_rows_of_the_twin():
    # the twin builds M from polynomials in e; the typed table must agree
    assert np.array_equal(L.M, BF.M_BF.astype(np.float64))


def test_storage_shift_moves_only_the_rho_e_zeta_moments():
    """The LB_BF16 step works on the stored shifted populations g = f - w rho_s: since
    M w = (1, -2, 1, 0, ..., 0), the moments of f are those of g plus rho_s (1, -2, 1) in
    rho, e and zeta, and M^-1 of m* less the same gives the shifted post-collision
    populations; f*_0 from mass conservation reads the same in shifted terms."""
    w36 = np.array([16, 4, 4, 4, 4, 1, 1, 1, 1], dtype=np.float64)      # 36 w, exact
    assert np.array_equal(L.M @ w36, np.array([36, -72, 36, 0, 0, 0, 0, 0, 0]))
    rng = np.random.default_rng(11)
    g = rng.normal(0.0, 0.05, size=9)
    rho_s = 0.37
    shift = np.array([1.0, -2.0, 1.0, 0, 0, 0, 0, 0, 0]) * rho_s
    assert np.allclose(L.M @ (g + W_EQ * rho_s), L.M @ g + shift, rtol=0, atol=1e-15)
    m_star = rng.normal(0.0, 0.1, size=9)
    f_star = L.M_INV @ m_star
    assert np.allclose(L.M_INV @ (m_star - shift), f_star - W_EQ * rho_s, rtol=0, atol=1e-15)
    rho = np.sum(g) + rho_s
    f0 = rho - np.sum(f_star[1:])                        # mass conservation, plain
    g0 = np.sum(g) - np.sum(f_star[1:] - W_EQ[1:] * rho_s)   # the same, shifted
    assert g0 == pytest.approx(f0 - W_EQ[0] * rho_s, abs=1e-14)


def test_equilibrium_moments_equal_m_times_textbook_feq():
    """Eq. 3 is M applied to the textbook D2Q9 equilibrium (checks every row of M and Eq. 3)."""
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.1, 3.0, size=(5, 6))
    ux, uy = rng.uniform(-0.3, 0.3, size=(2, 5, 6))
    meq = L.equilibrium_moments(rho, ux, uy)
    via_feq = np.tensordot(L.M, textbook_feq(rho, ux, uy), axes=(1, 0))
    assert np.allclose(meq, via_feq, rtol=0, atol=1e-14)


def test_forcing_moments_equal_m_times_guo_term():
    """Eq. 5 equals M applied to Guo's velocity-space forcing w_a[3(e-v).F + 9(e.v)(e.F)]."""
    rng = np.random.default_rng(4)
    vx, vy, Fx, Fy = rng.uniform(-0.2, 0.2, size=(4, 3, 4))
    guo = np.empty((9, 3, 4))
    for a, (ex, ey) in enumerate(E_VEC):
        ev = ex * vx + ey * vy
        guo[a] = W_EQ[a] * (3 * ((ex - vx) * Fx + (ey - vy) * Fy) + 9 * ev * (ex * Fx + ey * Fy))
    S = L.forcing_moments(vx, vy, Fx, Fy, np.ones_like(vx), 0.0, 0.8)
    assert np.allclose(S, np.tensordot(L.M, guo, axes=(1, 0)), rtol=0, atol=1e-15)


def test_sigma_term_enters_e_and_zeta_moments_only():
    """Eq. 8 adds 12 sigma |F|^2 / (psi^2 (tau_e - 1/2)) to S_1 and keeps S_2 = -S_1."""
    vx, vy, Fx, Fy, psi = (np.array([0.01]), np.array([-0.02]), np.array([0.003]),
                           np.array([0.004]), np.array([0.5]))
    s_e = 0.8
    S0 = L.forcing_moments(vx, vy, Fx, Fy, psi, 0.0, s_e)
    S1 = L.forcing_moments(vx, vy, Fx, Fy, psi, 0.1, s_e)
    d = (S1 - S0)[:, 0]
    expect = 12 * 0.1 * (0.003**2 + 0.004**2) / (0.25 * (1 / s_e - 0.5))
    assert d[1] == pytest.approx(expect, rel=1e-14)
    assert d[2] == pytest.approx(-expect, rel=1e-14)
    assert np.all(d[[0, 3, 4, 5, 6, 7, 8]] == 0)


def test_q_tensor_isotropy_identity():
    """sum_a w_a e_a e_a = I for w(1) = 1/3, w(2) = 1/12, so a linear psi gives Q_xy = 0
    and Qxx + Qyy vanishes for a harmonic psi (psi = x^2 - y^2)."""
    ny, nx = 12, 12
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    psi = 5.0 + 0.01 * (x - 6) ** 2 - 0.01 * (y - 6) ** 2
    nb = L.neighbour_psi(psi, False)
    Qxx, Qyy, Qxy = L.q_tensor(psi, nb, -1.0, 0.5)
    inner = (slice(2, -2), slice(2, -2))
    assert np.allclose((Qxx + Qyy)[inner], 0.0, atol=1e-15)
    assert np.allclose(Qxy[inner], 0.0, atol=1e-15)
    # only the two x-axis neighbours see the x-curvature (diagonal differences cancel):
    # Qxx = kappa G/2 psi * (1/3) * 2 * 0.01
    assert np.allclose(Qxx[inner], 0.5 * -1.0 / 2 * psi[inner] * 0.02 / 3, rtol=1e-12)


# ---------------------------------------------------------------- special cases

def test_bgk_limit_equals_textbook_bgk():
    """All rates equal and no force: MRT is BGK, f* = f - s (f - f_eq), then streaming."""
    rng = np.random.default_rng(5)
    rho = I.smooth_random_density(rng, 10, 9, 0.8, 1.2)
    f = I.random_populations(rng, rho)
    s = 1.3
    p = L.Params(eos=E.EOS(kind="exp"), G=0.0, rates=rates_all(s))
    out = L.step(f, p)
    r = f.sum(axis=0)
    ux = sum(ex * f[a] for a, (ex, ey) in enumerate(E_VEC)) / r
    uy = sum(ey * f[a] for a, (ex, ey) in enumerate(E_VEC)) / r
    fs = f - s * (f - textbook_feq(r, ux, uy))
    ref = np.empty_like(fs)
    ny, nx = r.shape
    for a, (ex, ey) in enumerate(E_VEC):
        for yy in range(ny):
            for xx in range(nx):
                ref[a, (yy + ey) % ny, (xx + ex) % nx] = fs[a, yy, xx]
    assert np.allclose(out, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("eos,G", [(E.cs_eos(0.8), -1.0), (E.EOS(kind="exp"), -40.0),
                                   (E.colosqui_eos(), -1.0)])
def test_uniform_state_is_stationary(eos, G):
    """Uniform rho at rest: F = Q = C = 0 exactly, so f stays at equilibrium."""
    rho0 = {"cs": 0.2, "exp": 300.0, "piecewise": 50.0}[eos.kind]
    rho = np.full((6, 7), rho0)
    f = L.equilibrium(rho, 0 * rho, 0 * rho)
    for walls in (False, True):
        p = L.Params(eos=eos, G=G, kappa=0.7, sigma_force=0.05, walls_y=walls)
        out = L.run(f, p, 20)
        assert np.allclose(out, f, rtol=1e-14, atol=0)


def test_shear_wave_decays_at_the_mrt_viscosity():
    """G = 0: u_x = U sin(2 pi y/N) decays as exp(-nu k^2 t), nu = (1/s_v - 1/2)/3."""
    N = 64
    rho, ux, uy = I.shear_wave(3, N, 1e-4)
    f = L.equilibrium(rho, ux, uy)
    for s_v in (1 / 0.8, 1.6):
        p = L.Params(eos=E.EOS(kind="exp"), G=0.0, rates=L.Rates(s_v=s_v))
        k, nu = 2 * np.pi / N, (1 / s_v - 0.5) / 3
        y = np.arange(N)
        g = L.run(f, p, 200)
        a0 = 2 * np.mean(L.macroscopic(g, p)[1][:, 0] * np.sin(k * y))
        g = L.run(g, p, 1000)
        a1 = 2 * np.mean(L.macroscopic(g, p)[1][:, 0] * np.sin(k * y))
        rate = np.log(a0 / a1) / 1000
        assert rate / (nu * k * k) == pytest.approx(1.0, abs=1e-3)


def test_mass_and_momentum_conserved_to_roundoff():
    """sum_x F = 0 on a periodic lattice (pair antisymmetry of Eq. 7) and C carries no
    mass or momentum, so total mass and bare momentum sum e f are invariants."""
    eos = E.cs_eos(0.8)
    rv, rl, _ = E.mechanical_stability(eos, -1.0)
    rng = np.random.default_rng(6)
    rho = I.droplet_density(40, 36, 10.0, rl, rv)
    ux, uy = I.random_velocity(rng, rho.shape, 0.01)
    f = L.equilibrium(rho, ux, uy)
    p = L.Params(eos=eos, G=-1.0, kappa=0.5, sigma_force=0.05, rates=L.Rates.from_viscosity(0.1))

    def totals(g):
        return g.sum(), sum(ex * g[a] for a, (ex, ey) in enumerate(E_VEC)).sum(), \
            sum(ey * g[a] for a, (ex, ey) in enumerate(E_VEC)).sum()

    m0, px0, py0 = totals(f)
    g = L.run(f, p, 300)
    m1, px1, py1 = totals(g)
    assert abs(m1 - m0) / m0 < 1e-13
    assert abs(px1 - px0) < 1e-12 * m0 and abs(py1 - py0) < 1e-12 * m0


# ---------------------------------------------------------------- brute-force twin

CASES = [
    (E.cs_eos(0.8), -1.0, 0.5, 0.0, (0.03, 0.30)),
    (E.cs_eos(0.9), -1.0, 0.3, 0.1, (0.05, 0.24)),
    (E.EOS(kind="exp"), -40.0, 0.7, 0.0, (85.0, 500.0)),
    (E.colosqui_eos(), -1.0, 0.5, 0.087, (1.0, 100.0)),
]


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_one_step_equals_bruteforce_twin(case, walls):
    eos, G, kappa, sigma, (lo, hi) = CASES[case]
    rng = np.random.default_rng(10 + case)
    rho = I.smooth_random_density(rng, 8, 7, lo, hi)
    f = I.random_populations(rng, rho)
    p = L.Params(eos=eos, G=G, kappa=kappa, sigma_force=sigma,
                 rates=L.Rates(s_rho=1.0, s_e=0.8, s_zeta=0.8, s_j=1.0, s_q=1.1, s_v=1.3),
                 walls_y=walls)
    a = L.step(f, p)
    b = BF.step(f, p).astype(np.float64)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()


@pytest.mark.parametrize("walls", [False, True])
def test_hundred_steps_equal_bruteforce_twin(walls):
    eos = E.cs_eos(0.8)
    rv, rl, _ = E.mechanical_stability(eos, -1.0)
    rho = I.droplet_density(8, 8, 2.5, rl, rv)
    f = L.equilibrium(rho, 0 * rho, 0 * rho)
    p = L.Params(eos=eos, G=-1.0, kappa=0.5, sigma_force=0.02,
                 rates=L.Rates.from_viscosity(0.1), walls_y=walls)
    a = L.run(f, p, 100)
    b = BF.run(f, p, 100).astype(np.float64)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_bounce_back_reflects_at_the_wall():
    """Half-way bounce-back: a population leaving row 0 downward comes back as its
    opposite at the same site one step later."""
    f = np.zeros((9, 4, 5))
    f[4, 0, 2] = 1.0                 # moving -y at the bottom row
    f[7, 3, 1] = 2.0                 # moving (-1, -1) ... not at the bottom: streams
    f[6, 3, 1] = 3.0                 # moving (-1, +1) at the top row: reflected as 8
    out = L.stream(f, walls_y=True)
    assert out[2, 0, 2] == 1.0
    assert out[7, 2, 0] == 2.0
    assert out[8, 3, 1] == 3.0
    assert out.sum() == 6.0


# ---------------------------------------------------------------- splash geometry (Sec. V.C)

def splash_params(case, switch=True):
    eos, G, kappa, sigma, (lo, hi) = CASES[case]
    rates = L.Rates(s_rho=1.0, s_e=0.8, s_zeta=0.8, s_j=1.0, s_q=1.1, s_v=1.6)
    sw = (0.5 * (lo + hi), 0.9) if switch else None
    return L.Params(eos=eos, G=G, kappa=kappa, sigma_force=sigma, rates=rates, open_bc=True,
                    visc_switch=sw), (lo, hi)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_open_boundaries_and_viscosity_switch_equal_bruteforce_twin(case):
    p, (lo, hi) = splash_params(case)
    rng = np.random.default_rng(40 + case)
    rho = I.smooth_random_density(rng, 8, 7, lo, hi)
    f = I.random_populations(rng, rho)
    a = L.step(f, p)
    b = BF.step(f, p).astype(np.float64)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()
    a = L.run(f, p, 20)
    b = BF.run(f, p, 20).astype(np.float64)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_viscosity_switch_limits_are_the_plain_rates():
    """rho_1 below every density: the liquid rate everywhere; above every density: the
    vapour rate everywhere."""
    p, (lo, hi) = splash_params(0)
    rng = np.random.default_rng(7)
    rho = I.smooth_random_density(rng, 16, 12, lo, hi)
    f = I.random_populations(rng, rho)
    low = L.Params(**{**p.__dict__, "visc_switch": (0.5 * lo, 0.9)})
    high = L.Params(**{**p.__dict__, "visc_switch": (2.0 * hi, 0.9)})
    liquid = L.Params(**{**p.__dict__, "visc_switch": None})
    vapour = L.Params(**{**p.__dict__, "visc_switch": None,
                         "rates": L.Rates(**{**p.rates.__dict__, "s_v": 0.9})})
    assert np.array_equal(L.step(f, low), L.step(f, liquid))
    assert np.array_equal(L.step(f, high), L.step(f, vapour))
    assert not np.allclose(L.step(f, p), L.step(f, liquid))


def test_open_boundary_rest_state_is_stationary():
    eos = E.cs_eos(0.8)
    f = L.equilibrium(np.full((9, 11), 0.2), np.zeros((9, 11)), np.zeros((9, 11)))
    p = L.Params(eos=eos, G=-1.0, kappa=0.3, open_bc=True, visc_switch=(0.1, 0.9))
    assert np.abs(L.run(f, p, 50) - f).max() < 1e-15


def test_open_sides_equal_periodic_for_states_uniform_in_x():
    """Zero-gradient side boundaries see the same neighbour values as periodic ones when
    nothing depends on x; the top row then differs only through the open top."""
    eos = E.cs_eos(0.8)
    rv, rl, _ = E.mechanical_stability(eos, -1.0)
    ny, nx = 24, 10
    rho = I.layer_density(nx, ny, 10.0, rl, rv, width=3.0)
    f = L.equilibrium(rho, 0 * rho, 0 * rho)
    p_open = L.Params(eos=eos, G=-1.0, kappa=0.5, open_bc=True)
    p_walls = L.Params(eos=eos, G=-1.0, kappa=0.5, walls_y=True)
    a = L.run(f, p_open, 5)
    b = L.run(f, p_walls, 5)
    assert np.allclose(a, a[:, :, :1], atol=1e-15, rtol=0)       # stays uniform in x
    # one step reaches two rows (pull, then psi of the neighbours): after 5 steps the rows
    # more than 10 below the top, where open and wall boundaries differ, agree to round-off
    assert np.abs(a[:, :ny - 11] - b[:, :ny - 11]).max() < 1e-13
    assert np.abs(a[:, ny - 1] - b[:, ny - 1]).max() > 1e-10   # the boundaries do differ


def test_open_boundary_pull_copies_the_nearest_site():
    f = np.zeros((9, 4, 5))
    f[1, 2, 0] = 1.0           # +x population at the left column: also pulled into x = 0
    f[4, 3, 2] = 2.0           # -y population at the top row: pulled from the top row itself
    f[4, 0, 3] = 5.0           # -y population at the bottom row: bounced back as +y
    out = L.stream(f, walls_y=False, open_bc=True)
    assert out[1, 2, 0] == 1.0 and out[1, 2, 1] == 1.0
    assert out[4, 3, 2] == 2.0 and out[4, 2, 2] == 2.0
    assert out[2, 0, 3] == 5.0
