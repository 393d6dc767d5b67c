"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances
----------
FP64: the GPU evaluates the same per-site formulas in a different association order and
with fused multiply-adds, so a step differs by a few ulps of the largest moment; over
many damped steps the difference stays near 1e-14 relative. Bar: 1e-13 relative for up
to 10 steps, 1e-11 relative density per site after the 5000-step droplet.

FP32: unit roundoff u = 2^-24 ~ 6e-8. One step evaluates m = M f, the relaxation and
f* = M^-1 m* in about 40 dependent operations on values bounded by |m| <= 4 rho_max,
and psi through an EOS with one division and one square root; a forward error bound of
the order 60 u rho_max ~ 4e-6 rho_max per step covers it, and the map is non-expansive
(|1 - s| < 1), so errors add at most linearly over steps. Bar: 5e-6 * n_steps relative to
max |f|.
"""
import zlib

import numpy as np
import pytest

from oracle import eos as OE
from oracle import lattice as OL
from paper_1306_6445_gb300 import inputs as I

from _util import oracle_params, rel_err, window

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_6445_gb300 import _build

    _build.build()
    from paper_1306_6445_gb300 import lbm as mod

    mod.load_library()
    return mod


def case_params(lbm, kind):
    if kind == "cs":
        return lbm.cs_eos(0.8), -1.0, (0.02, 0.31)
    if kind == "exp":
        return lbm.EOSParams(kind="exp"), -40.0, (150.0, 420.0)
    return lbm.EOSParams(kind="piecewise"), -1.0, (1.0, 100.0)


def fp32_tol(n):
    return 5e-6 * n


# --------------------------------------------------------------------------- element-wise

SIZES = [(3, 3), (8, 8), (37, 29), (129, 67), (200, 136), (300, 9)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("kind", ["cs", "exp", "piecewise"])
@pytest.mark.parametrize("size", SIZES)
def test_steps_match_oracle_elementwise(lbm, prec, walls, kind, size):
    nx, ny = size
    eos, G, (lo, hi) = case_params(lbm, kind)
    kappa, sigma = 0.6, (0.087 if kind == "piecewise" else 0.05)
    rates = lbm.RateParams(s_rho=1.0, s_e=0.8, s_zeta=0.8, s_j=1.2, s_q=1.1, s_v=1.3)
    rng = np.random.default_rng(zlib.crc32(repr((nx, ny, kind, walls)).encode()))
    rho = I.smooth_random_density(rng, nx, ny, lo, hi)
    f0 = I.random_populations(rng, rho)
    lat = lbm.Lattice(nx, ny, eos, G, kappa=kappa, sigma_force=sigma, rates=rates, prec=prec,
                      walls_y=walls)
    lat.set_populations(f0)
    f0 = f0.astype(lat.dtype).astype(np.float64)   # the values the GPU holds (storage type)
    p = oracle_params(eos, G, kappa, sigma, rates, walls)
    n = 1 if max(nx, ny) > 150 else 4
    lat.step(n)
    got = lat.populations()
    lat.close()
    ref = OL.run(f0, p, n)
    tol = 1e-13 if prec == "fp64" else fp32_tol(n)
    assert rel_err(got, ref) <= tol


def test_equilibrium_initialisation_matches_oracle(lbm):
    eos, G, _ = case_params(lbm, "cs")
    nx, ny = 50, 41
    rho = I.droplet_density(nx, ny, 12.0, 0.31, 0.02)
    ux, uy = I.random_velocity(np.random.default_rng(2), rho.shape, 0.05)
    lat = lbm.Lattice(nx, ny, eos, G, prec="fp64")
    lat.set_rho_u(rho, ux, uy)
    got = lat.populations()
    assert rel_err(got, OL.equilibrium(rho, ux, uy)) < 1e-15
    assert lat.steps_done == 0
    lat.close()


# --------------------------------------------------------------------------- the c0 run

@pytest.mark.parametrize("kappa", [0.0, 0.5])
def test_droplet_128_fp64_5000_steps_density_parity(lbm, kappa):
    """128^2 periodic droplet, CS at 0.8 T_c, G = -1, nu = 0.1, R = 30, tanh width 2,
    Maxwell densities: rho per site after 5000 steps within 1e-11 relative."""
    eos = lbm.cs_eos(0.8)
    rv, rl, _ = lbm.lb_maxwell(eos, -1.0)
    rates = lbm.RateParams.from_viscosity(0.1)
    rho = I.droplet_density(128, 128, 30.0, rl, rv)
    lat = lbm.Lattice(128, 128, eos, -1.0, kappa=kappa, rates=rates, prec="fp64")
    lat.set_rho_u(rho)
    f0 = lat.populations()
    m0 = lat.reduce()
    lat.step(5000)
    got_rho = lat.rho()
    m1 = lat.reduce()
    lat.close()
    p = oracle_params(eos, -1.0, kappa, 0.0, rates)
    ref = OL.run(f0, p, 5000)
    ref_rho = OL.density(ref)
    assert np.max(np.abs(got_rho - ref_rho) / ref_rho) <= 1e-11
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-12          # mass conservation on the GPU


# --------------------------------------------------------------------------- full size

def sampled_sites(nx, ny, rng, n=48, walls=False):
    xs = list(rng.integers(0, nx, size=n)) + [0, nx - 1, 127, 128, 0, nx - 1]
    ys = list(rng.integers(0, ny, size=n)) + [0, ny - 1, 0, ny - 1, ny // 2, ny // 2]
    return list(zip(xs, ys))


@pytest.mark.parametrize("prec,nx,ny,walls", [("fp32", 2048, 2048, False),
                                              ("fp64", 2048, 2048, False),
                                              ("fp32", 4096, 2048, True)])
def test_full_size_step_sampled_against_oracle(lbm, prec, nx, ny, walls):
    """At the benchmark sizes and launch configuration: one step from a droplet state with
    random velocities; sampled sites (plus lattice and tile edges) are recomputed by the
    oracle from their 5x5 neighbourhood."""
    eos = lbm.cs_eos(0.8)
    rv, rl, _ = lbm.lb_maxwell(eos, -1.0)
    rates = lbm.RateParams.from_viscosity(0.1)
    rng = np.random.default_rng(77)
    if walls:
        rho = I.layer_density(nx, ny, ny / 2, rl, rv, amplitude=0.01 * nx, wavenumber=1)
    else:
        rho = I.droplet_density(nx, ny, 200.0, rl, rv)
    ux, uy = I.random_velocity(rng, rho.shape, 0.02)
    lat = lbm.Lattice(nx, ny, eos, -1.0, kappa=0.6, sigma_force=0.02, rates=rates, prec=prec,
                      walls_y=walls)
    lat.set_rho_u(rho, ux, uy)
    lat.autotune(3)                  # the launch the benchmark would choose
    f0 = lat.populations().astype(np.float64)
    lat.step(1)
    got = lat.populations()
    lat.close()
    p = oracle_params(eos, -1.0, 0.6, 0.02, rates, walls)
    tol = 1e-13 if prec == "fp64" else fp32_tol(1)
    scale = np.abs(f0).max()
    for (x, y) in sampled_sites(nx, ny, rng, walls=walls):
        sub, cx, cy, sw = window(f0, x, y, walls)
        pp = oracle_params(eos, -1.0, 0.6, 0.02, rates, sw)
        ref = OL.step(sub, pp)[:, cy, cx]
        assert np.abs(got[:, y, x] - ref).max() <= tol * scale, (x, y)
    del p


# --------------------------------------------------------------------------- diagnostics

def test_rho_u_and_reduction_match_oracle(lbm):
    eos, G, _ = case_params(lbm, "cs")
    rates = lbm.RateParams.from_viscosity(0.1)
    nx, ny = 96, 70
    rho = I.droplet_density(nx, ny, 20.0, 0.31, 0.02)
    ux, uy = I.random_velocity(np.random.default_rng(3), rho.shape, 0.01)
    lat = lbm.Lattice(nx, ny, eos, G, kappa=0.3, rates=rates, prec="fp64", walls_y=True)
    lat.set_rho_u(rho, ux, uy)
    lat.step(25)
    f = lat.populations()
    p = oracle_params(eos, G, 0.3, 0.0, rates, True)
    r, vx, vy = OL.macroscopic(f, p)
    assert rel_err(lat.rho(), r) < 1e-15
    gx, gy = lat.u()
    assert np.abs(gx - vx).max() < 1e-15 and np.abs(gy - vy).max() < 1e-15
    red = lat.reduce()
    assert red[0] == pytest.approx(r.sum(), rel=1e-13)
    assert red[1] == pytest.approx((r * vx).sum(), abs=1e-13 * r.sum())
    assert red[2] == pytest.approx((r * vy).sum(), abs=1e-13 * r.sum())
    assert red[3] == pytest.approx(np.sqrt(vx**2 + vy**2).max(), rel=1e-14)
    # fixed reduction order: identical bits on repeat
    assert np.array_equal(red, lat.reduce())
    lat.close()


def test_checkpoint_resume_is_bit_identical(lbm):
    eos, G, _ = case_params(lbm, "exp")
    rates = lbm.RateParams.from_viscosity(0.1)
    rho = I.droplet_density(64, 48, 12.0, 515.0, 80.0)
    for prec in ("fp32", "fp64"):
        lat = lbm.Lattice(64, 48, eos, G, kappa=0.5, rates=rates, prec=prec)
        lat.set_rho_u(rho)
        lat.step(20)
        ck = lat.populations()
        lat.step(20)
        a = lat.populations()
        lat.set_populations(ck)
        lat.step(20)
        b = lat.populations()
        assert np.array_equal(a, b)
        lat.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("bc", ["periodic", "walls", "open"])
def test_page_locked_and_pageable_host_buffers_give_the_same_bits(lbm, prec, bc):
    """lb_get_populations, lb_set_populations and lb_get_rho give the same bits with
    page-locked host buffers (the bench's end-to-end path) as with pageable ones."""
    if prec == "bf16" and bc == "open":
        pytest.skip("open boundaries are not compiled for BF16 storage")
    eos, G, _ = case_params(lbm, "cs")
    rv, rl, _ = lbm.lb_maxwell(eos, G)
    kw = {"walls_y": True} if bc == "walls" else ({"open_bc": True} if bc == "open" else {})
    nx, ny = 131, 67
    mk = lambda: lbm.Lattice(nx, ny, eos, G, kappa=0.3, rates=lbm.RateParams.from_viscosity(0.1),
                             prec=prec, storage_shift=rv, **kw)
    lat = mk()
    lat.set_rho_u(I.droplet_density(nx, ny, 15.0, rl, rv))
    lat.step(7)
    tdt = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.int16}[prec]
    pinned = torch.empty((9, ny, nx), dtype=tdt, pin_memory=True)
    lbm.lb_get_populations(lat.ctx, pinned.data_ptr(), pinned.numel() * pinned.element_size())
    f_pageable = lat.populations()
    assert np.array_equal(pinned.numpy().view(f_pageable.dtype), f_pageable)
    rho_pinned = torch.empty((ny, nx), dtype=torch.float64, pin_memory=True).numpy()
    lbm.lb_get_rho(lat.ctx, rho_pinned)
    assert np.array_equal(rho_pinned, lat.rho())
    lat.close()
    outs = []
    for src in ("pinned", "pageable"):
        b = mk()
        if src == "pinned":
            lbm.lb_set_populations(b.ctx, pinned.data_ptr(), pinned.numel() * pinned.element_size())
        else:
            b.set_populations(f_pageable)
        b.step(3)
        outs.append(b.populations())
        b.close()
    assert np.array_equal(outs[0], outs[1])


def test_library_owned_buffers_and_default_stream(lbm):
    eos, G, _ = case_params(lbm, "exp")
    rho = I.droplet_density(40, 40, 10.0, 515.0, 80.0)
    a = lbm.Lattice(40, 40, eos, G, kappa=0.2, prec="fp64", buffers="library")
    b = lbm.Lattice(40, 40, eos, G, kappa=0.2, prec="fp64", buffers="torch")
    for lat in (a, b):
        lat.set_rho_u(rho)
        lat.step(7)
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()


# --------------------------------------------------------------------------- errors

def test_domain_error_at_initialisation(lbm):
    eos = lbm.cs_eos(0.8)
    rho = np.full((16, 16), 0.2)
    rho[3, 4] = 0.7      # (p - rho/3)/G < 0 above ~0.47 for CS at 0.8 T_c, G = -1
    lat = lbm.Lattice(16, 16, eos, -1.0, prec="fp32")
    with pytest.raises(lbm.LBError) as ei:
        lat.set_rho_u(rho)
    assert ei.value.status == lbm.LB_EDOMAIN
    # poisoned: later calls report the same status
    with pytest.raises(lbm.LBError) as ei:
        lat.step(1)
    assert ei.value.status == lbm.LB_EDOMAIN
    lat.close()


def test_domain_error_found_during_stepping(lbm):
    eos = lbm.cs_eos(0.8)
    f = np.zeros((9, 12, 12))
    f[0] = 0.2
    f[0, 5, 5] = -0.1    # negative density at one site (host-made bad input)
    lat = lbm.Lattice(12, 12, eos, -1.0, prec="fp64")
    lat.set_populations(f)
    lat.step(2)
    with pytest.raises(lbm.LBError) as ei:
        lat.sync()
    assert ei.value.status == lbm.LB_EDOMAIN
    lat.close()


def test_nonfinite_reduction_poisons_the_context(lbm):
    eos = lbm.EOSParams(kind="exp")
    f = np.zeros((9, 8, 8))
    f[0] = 300.0
    f[1, 2, 2], f[3, 2, 2] = 1e308, -1e308     # finite rho, overflowing momentum
    lat = lbm.Lattice(8, 8, eos, -40.0, prec="fp64")
    lat.set_populations(f)
    with pytest.raises(lbm.LBError) as ei:
        lat.reduce()
    assert ei.value.status == lbm.LB_ENONFINITE
    with pytest.raises(lbm.LBError):
        lat.rho()
    lat.close()


def test_size_mismatch_is_einval(lbm):
    lat = lbm.Lattice(10, 10, lbm.EOSParams(kind="exp"), -40.0, prec="fp64")
    buf = np.zeros((9, 10, 9))
    with pytest.raises(lbm.LBError) as ei:
        lbm.lb_set_populations(lat.ctx, buf.ctypes.data, buf.nbytes)
    assert ei.value.status == lbm.LB_EINVAL
    lat.close()


def test_zero_steps_is_a_no_op(lbm):
    eos, G, _ = case_params(lbm, "exp")
    rho = I.droplet_density(20, 20, 5.0, 515.0, 80.0)
    lat = lbm.Lattice(20, 20, eos, G, prec="fp64")
    lat.set_rho_u(rho)
    a = lat.populations()
    lat.step(0)
    assert np.array_equal(a, lat.populations())
    lat.close()


# --------------------------------------------------------------------------- launch shapes

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_every_launch_variant_gives_identical_bits(lbm, prec):
    """The per-site arithmetic does not depend on the strip width, ring depth or rows per
    CTA, so every launch shape must produce the same bits (and match the oracle)."""
    eos, G, (lo, hi) = case_params(lbm, "cs")
    rates = lbm.RateParams.from_viscosity(0.1)
    nx, ny = 301, 77
    rng = np.random.default_rng(5)
    rho = I.smooth_random_density(rng, nx, ny, lo, hi)
    f0 = I.random_populations(rng, rho)
    results = []
    for walls in (False, True):
        # rows 19 and 25 leave a last row block of 1 and 2 rows (77 = 4 x 19 + 1 = 3 x 25 + 2)
        shapes = [(v, r) for v in range(lbm.lb_launch_variants()) for r in (0, 8, 13, 19, 25, 77)]
        outs = []
        for (v, r) in shapes:
            lat = lbm.Lattice(nx, ny, eos, G, kappa=0.4, sigma_force=0.05, rates=rates,
                              prec=prec, walls_y=walls)
            lbm.lb_set_launch(lat.ctx, v, r)
            lat.set_populations(f0)
            lat.step(3)
            outs.append(lat.populations())
            lat.close()
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
        p = oracle_params(eos, G, 0.4, 0.05, rates, walls)
        ref = OL.run(f0.astype(prec == "fp32" and np.float32 or np.float64).astype(np.float64), p, 3)
        tol = 1e-13 if prec == "fp64" else fp32_tol(3)
        assert rel_err(outs[0], ref) <= tol
        results.append(outs[0])


@pytest.mark.parametrize("walls", [False, True])
def test_autotune_keeps_the_state_and_the_bits(lbm, walls):
    """lb_autotune only writes the spare buffer: the state and step count are unchanged,
    and stepping after it gives the same bits as the default launch."""
    eos, G, (lo, hi) = case_params(lbm, "cs")
    rates = lbm.RateParams.from_viscosity(0.1)
    nx, ny = 517, 203
    rng = np.random.default_rng(11)
    rho = I.smooth_random_density(rng, nx, ny, lo, hi)
    f0 = I.random_populations(rng, rho)
    outs = []
    for tune in (False, True):
        lat = lbm.Lattice(nx, ny, eos, G, kappa=0.3, sigma_force=0.05, rates=rates,
                          prec="fp32", walls_y=walls)
        lat.set_populations(f0)
        lat.step(2)
        if tune:
            before = lat.populations()
            v, r = lat.autotune(2)
            assert 0 <= v < lbm.lb_launch_variants() and 1 <= r <= ny
            assert lbm.lb_get_launch(lat.ctx)["variant"] == v
            assert np.array_equal(lat.populations(), before) and lat.steps_done == 2
        lat.step(5)
        outs.append(lat.populations())
        lat.close()
    assert np.array_equal(outs[0], outs[1])


def test_stalled_wait_times_out_and_poisons(lbm):
    """A ring row that is never requested makes the bounded mbarrier wait give up after
    about a second: the step reports LB_ETIMEOUT instead of hanging, and later calls keep
    returning it."""
    eos = lbm.EOSParams(kind="exp")
    rho = I.droplet_density(64, 64, 12.0, 400.0, 150.0)
    lat = lbm.Lattice(64, 64, eos, -40.0, prec="fp32")
    lat.set_rho_u(rho)
    lbm.lb_debug_stall_row(lat.ctx, 20)
    lat.step(1)
    with pytest.raises(lbm.LBError) as ei:
        lat.sync()
    assert ei.value.status == lbm.LB_ETIMEOUT
    with pytest.raises(lbm.LBError) as ei:
        lat.step(1)
    assert ei.value.status == lbm.LB_ETIMEOUT
    lat.close()
    # the device is still usable afterwards
    lat = lbm.Lattice(16, 16, eos, -40.0, prec="fp32")
    lat.set_rho_u(np.full((16, 16), 300.0))
    lat.step(2)
    assert np.allclose(lat.rho(), 300.0, rtol=1e-6)
    lat.close()
