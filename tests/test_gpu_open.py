"""LB_BC_OPEN (bounce-back wall below, zero-gradient open boundaries above and at the sides)
with the density-dependent viscosity of Sec. V.C, on the GPU against the FP64 oracle.

Initial states are made consistent with the open boundaries by the oracle's own streaming
(f0 = pull of a random post-collision field), so the GPU holds exactly f0 after
lb_set_populations. The switch density rho_1 is placed in a gap of the densities of every
step of the oracle's run, so that the two sides take the same rate at every site (the
GPU decides in its own precision)."""
import zlib

import numpy as np
import pytest

from oracle import lattice as OL
from paper_1306_6445_gb300 import inputs as I

from _util import oracle_params, rel_err

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


def switch_density(trajs, near):
    """The middle of the widest-enough gap (> 2e-4 relative) nearest `near` among the
    densities of every trajectory given."""
    vals = np.sort(np.concatenate([OL.density(f).ravel() for t in trajs for f in t]))
    big = np.flatnonzero(np.diff(vals) > 2e-4 * near)
    i = int(big[np.argmin(np.abs(vals[big] - near))])
    return 0.5 * (vals[i] + vals[i + 1])


def switched_run(f0, p_of, n, lo, hi):
    """rho_1 and the oracle trajectory with the switch there, such that no density of the
    trajectory lies within 1e-4 of rho_1 (so FP32 and FP64 put every site on the same
    side). The switch changes the trajectory, so the choice is repeated until it holds."""
    trajs = []
    r1 = 0.5 * (lo + hi)
    for _ in range(8):
        traj = [f0]
        p = p_of(r1)
        for _ in range(n):
            traj.append(OL.step(traj[-1], p))
        trajs.append(traj[:-1])
        d = min(np.min(np.abs(OL.density(f) - r1)) for f in traj[:-1])
        if d > 1e-4 * r1:
            return r1, traj[-1]
        r1 = switch_density(trajs, r1)
    raise AssertionError("no switch density clear of the trajectory")


def consistent_state(rng, nx, ny, lo, hi):
    rho = I.smooth_random_density(rng, nx, ny, lo, hi)
    return OL.stream(I.random_populations(rng, rho), walls_y=False, open_bc=True)


SIZES = [(8, 8), (37, 29), (129, 67), (300, 9)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["cs", "exp", "piecewise"])
@pytest.mark.parametrize("size", SIZES)
def test_open_boundaries_and_viscosity_switch_match_oracle(lbm, prec, kind, size):
    nx, ny = size
    eos, G, (lo, hi) = case_params(lbm, kind)
    kappa, sigma = 0.6, (0.087 if kind == "piecewise" else 0.05)
    rates = lbm.RateParams(s_rho=1.0, s_e=0.8, s_zeta=0.8, s_j=1.2, s_q=1.1, s_v=1.7)
    rng = np.random.default_rng(zlib.crc32(repr(("open", nx, ny, kind)).encode()))
    f0 = consistent_state(rng, nx, ny, lo, hi).astype(np.float32 if prec == "fp32" else np.float64)
    f0 = f0.astype(np.float64)
    n = 4

    def p_of(r1):
        return oracle_params(eos, G, kappa, sigma, rates, open_bc=True, visc_switch=(r1, 0.9))

    r1, ref = switched_run(f0, p_of, n, lo, hi)
    lat = lbm.Lattice(nx, ny, eos, G, kappa=kappa, sigma_force=sigma, rates=rates, prec=prec,
                      open_bc=True, viscosity_switch=(r1, 0.9))
    lat.set_populations(f0)
    assert np.array_equal(lat.populations().astype(np.float64), f0)   # f0 is representable
    lat.step(n)
    got = lat.populations()
    lat.close()
    tol = 1e-13 if prec == "fp64" else 5e-6 * n
    assert rel_err(got, ref) <= tol


def test_every_launch_variant_gives_identical_bits(lbm):
    eos, G, (lo, hi) = case_params(lbm, "piecewise")
    rates = lbm.RateParams.from_viscosity(0.0125)
    f0 = consistent_state(np.random.default_rng(3), 301, 77, lo, hi)
    outs = []
    for v in range(lbm.lb_launch_variants()):
        for r in (0, 9):
            lat = lbm.Lattice(301, 77, eos, G, kappa=0.3, sigma_force=0.087, rates=rates,
                              prec="fp32", open_bc=True, viscosity_switch=(1.49, 0.8))
            lbm.lb_set_launch(lat.ctx, v, r)
            lat.set_populations(f0)
            lat.step(5)
            outs.append(lat.populations())
            lat.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_checkpoint_resume_is_bit_identical(lbm):
    eos, G, (lo, hi) = case_params(lbm, "cs")
    rates = lbm.RateParams.from_viscosity(0.1)
    rho = I.droplet_density(96, 64, 15.0, hi, lo)
    kw = dict(kappa=0.5, rates=rates, prec="fp32", open_bc=True, viscosity_switch=(0.1, 1.0))
    a = lbm.Lattice(96, 64, eos, G, **kw)
    a.set_rho_u(rho)
    a.step(30)
    b = lbm.Lattice(96, 64, eos, G, **kw)
    b.set_populations(a.populations())
    a.step(25)
    b.step(25)
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()


def test_argument_errors(lbm):
    eos = lbm.cs_eos(0.8)
    with pytest.raises(lbm.LBError):
        lbm.Lattice(32, 32, eos, -1.0, prec="bf16", open_bc=True)
    per = lbm.Lattice(32, 32, eos, -1.0, prec="fp32")
    with pytest.raises(lbm.LBError):
        lbm.lb_set_viscosity_switch(per.ctx, 0.1, 0.9)
    per.close()
    op = lbm.Lattice(32, 32, eos, -1.0, prec="fp32", open_bc=True)
    with pytest.raises(lbm.LBError):
        lbm.lb_set_viscosity_switch(op.ctx, 0.1, 2.5)
    op.set_rho_u(np.full((32, 32), 0.1))
    with pytest.raises(lbm.LBError):
        lbm.lb_reduce_noalloc(op.ctx)
    m = op.reduce()
    assert np.isfinite(m).all()
    op.close()
