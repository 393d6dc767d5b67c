"""Batched lattices (lb_batch_*) on the GPU: every lattice of a batch evolves bit for bit
like the same lattice run alone through lb_step (so the oracle parity of the single path
carries over), the persistent launch and the graph replay agree with direct launches, the
GPU Laplace sums equal sums recomputed on the host from the same densities, one failing
lattice does not stop the others, and the autotuner returns a working launch."""
import numpy as np
import pytest

from oracle import diagnostics as D
from paper_1306_6445_gb300 import inputs as I

from _util import oracle_params

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


def small_batch(lbm):
    """Uneven sizes (ragged, narrower and wider than one strip), temperatures, kappa, tau."""
    specs = [(64, 64, 0.80, 0.0, 0.8), (96, 80, 0.70, 0.5, 0.6), (130, 70, 0.90, 0.3, 1.0),
             (160, 160, 0.65, 0.9, 1.2), (257, 131, 0.85, 0.6, 0.7), (33, 40, 0.75, 0.2, 0.9)]
    descs, rhos, radii = [], [], []
    for (nx, ny, t, kappa, tau) in specs:
        eos = lbm.cs_eos(t)
        rv, rl, _ = lbm.lb_maxwell(eos, -1.0)
        rates = lbm.RateParams(s_v=1.0 / tau)
        descs.append(lbm.LatticeDesc(nx, ny, eos, -1.0, kappa=kappa, sigma_force=0.087,
                                     rates=rates))
        R = 0.25 * min(nx, ny)
        radii.append(R)
        rhos.append(I.droplet_density(nx, ny, R, rl, rv))
    return descs, rhos, np.array(radii)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_equals_single_lattice_runs_bitwise(lbm, prec):
    descs, rhos, _ = small_batch(lbm)
    b = lbm.Batch(descs, prec=prec)
    for i, r in enumerate(rhos):
        b.set_rho_u(i, r)
    steps = 64 + 7          # one graph replay plus direct launches
    b.step(steps)
    b.sync()
    for i, d in enumerate(descs):
        lat = lbm.Lattice(d.nx, d.ny, d.eos, d.G, kappa=d.kappa, sigma_force=d.sigma_force,
                          rates=d.rates, prec=prec)
        lat.set_rho_u(rhos[i])
        lat.step(steps)
        assert np.array_equal(b.populations(i), lat.populations()), i
        lat.close()
    assert b.steps_done == steps
    assert not b.errors().any()
    b.close()


def test_batch_launch_shapes_and_autotune_agree(lbm):
    descs, rhos, _ = small_batch(lbm)
    outs = []
    for shape in [(0, 16), (1, 8), (2, 12), (3, 24), (4, 12), (5, 8), (6, 16), None]:
        b = lbm.Batch(descs, prec="fp32")
        if shape is not None:
            b.set_launch(*shape)
        for i, rr in enumerate(rhos):
            b.set_rho_u(i, rr)
        b.step(5)
        if shape is None:
            # timed on the current states, which it restores with the step count
            before = [b.populations(i) for i in range(len(descs))]
            v, r = b.autotune(3)
            assert 0 <= v < lbm.lb_launch_variants() and r > 0
            assert b.steps_done == 5
            for i in range(len(descs)):
                assert np.array_equal(b.populations(i), before[i])
        b.step(15)
        outs.append([b.populations(i) for i in range(len(descs))])
        b.close()
    for o in outs[1:]:
        for a, c in zip(o, outs[0]):
            assert np.array_equal(a, c)


def test_batch_measure_matches_host_sums(lbm):
    descs, rhos, radii = small_batch(lbm)
    b = lbm.Batch(descs, prec="fp64")
    for i, r in enumerate(rhos):
        b.set_rho_u(i, r)
    b.step(300)
    m = b.measure(radii)
    for i, d in enumerate(descs):
        rho = b.rho(i)
        p = oracle_params(d.eos, d.G, d.kappa, d.sigma_force, d.rates)
        from oracle import lattice as OL
        pres = OL.pressure(rho, p)
        y, x = np.mgrid[0:d.ny, 0:d.nx].astype(float)
        r = np.hypot(x - (d.nx - 1) / 2, y - (d.ny - 1) / 2)
        inside = r < radii[i] / 2
        outside = r > radii[i] + 0.3 * min(d.nx, d.ny) / 2
        rho_in, rho_out = rho[inside].mean(), rho[outside].mean()
        p_in, p_out = pres[inside].mean(), pres[outside].mean()
        R = np.sqrt((rho.sum() - rho_out * rho.size) / (np.pi * (rho_in - rho_out)))
        assert m[i, 1] == pytest.approx(rho_in, rel=1e-12)
        assert m[i, 2] == pytest.approx(rho_out, rel=1e-12)
        assert m[i, 4] == pytest.approx(p_in, rel=1e-10)
        assert m[i, 5] == pytest.approx(p_out, rel=1e-10)
        assert m[i, 3] == pytest.approx(R, rel=1e-10)
        assert m[i, 0] == pytest.approx((p_in - p_out) * R, rel=1e-8, abs=1e-12)
        assert m[i, 7] == 0
    b.close()


def test_batch_measure_agrees_with_oracle_laplace_on_converged_droplets(lbm):
    """The GPU measurement and the oracle's Laplace reading (which locates the droplet from
    the field itself) agree on converged droplets."""
    eos = lbm.EOSParams(kind="piecewise")
    descs = [lbm.LatticeDesc(96, 96, eos, -1.0, kappa=k, sigma_force=0.087,
                             rates=lbm.RateParams.from_viscosity(0.1)) for k in (0.0, 0.5)]
    b = lbm.Batch(descs, prec="fp64")
    for i in range(2):
        b.set_rho_u(i, I.droplet_density(96, 96, 28.0, 100.0, 1.0))
    b.step(20000)
    m = b.measure(np.array([28.0, 28.0]))
    for i, d in enumerate(descs):
        ref = D.laplace(b.rho(i), oracle_params(d.eos, d.G, d.kappa, d.sigma_force, d.rates))
        assert m[i, 0] == pytest.approx(ref["theta"], rel=0.01)
        assert m[i, 1] == pytest.approx(ref["rho_in"], rel=1e-4)
        assert m[i, 2] == pytest.approx(ref["rho_out"], rel=2e-3)
    assert m[1, 0] / m[0, 0] == pytest.approx(0.5, abs=0.02)
    b.close()


def test_a_failing_lattice_is_flagged_and_the_others_continue(lbm):
    descs, rhos, radii = small_batch(lbm)
    b = lbm.Batch(descs, prec="fp32")
    for i, r in enumerate(rhos):
        b.set_rho_u(i, r)
    # a density far outside the CS branch at one site of lattice 2 (host-made bad input)
    bad = rhos[2].copy()
    bad[10, 10] = 0.6
    with pytest.raises(lbm.LBError) as ei:
        b.set_rho_u(2, bad)
    assert ei.value.status == lbm.LB_EDOMAIN
    b.step(10)
    flags = b.errors()
    assert flags[2] != 0 and not np.delete(flags, 2).any()
    m = b.measure(radii)
    assert m[2, 7] == 1 and not m[np.arange(len(descs)) != 2, 7].any()
    b.close()


def single_run(lbm, d, rho, steps, prec="fp32"):
    lat = lbm.Lattice(d.nx, d.ny, d.eos, d.G, kappa=d.kappa, sigma_force=d.sigma_force,
                      rates=d.rates, prec=prec)
    lat.set_rho_u(rho)
    lat.step(steps)
    out = lat.populations()
    lat.close()
    return out


def test_inactive_lattices_keep_their_state_and_can_resume(lbm):
    """lb_batch_set_active: an inactive lattice is not advanced, keeps its state (readable
    and measurable at any step count), and continues like a lattice that was never
    stopped once made active again; the active ones are unaffected."""
    descs, rhos, radii = small_batch(lbm)
    b = lbm.Batch(descs, prec="fp32")
    for i, r in enumerate(rhos):
        b.set_rho_u(i, r)
    b.step(64)
    frozen = [1, 4]
    snap = {i: b.populations(i) for i in frozen}
    m_before = b.measure(radii)
    active = np.ones(len(descs), dtype=bool)
    active[frozen] = False
    b.set_active(active)
    b.step(64 + 3)                       # graph replay, then direct launches: odd count
    assert b.steps_done == 131
    for i in range(len(descs)):
        assert b.lattice_steps(i) == (64 if i in frozen else 131)
    # readable and measurable while the batch's step count is odd
    m_odd = b.measure(radii)
    for i in frozen:
        assert np.array_equal(b.populations(i), snap[i])
        assert np.array_equal(m_odd[i], m_before[i])
    for i in range(len(descs)):
        if i not in frozen:
            assert np.array_equal(b.populations(i), single_run(lbm, descs[i], rhos[i], 131)), i
    # changing the set at an odd step count is refused and changes nothing
    with pytest.raises(lbm.LBError) as ei:
        b.set_active(np.ones(len(descs), dtype=bool))
    assert ei.value.status == lbm.LB_EINVAL
    b.step(1)                            # even again
    b.set_active(np.ones(len(descs), dtype=bool))
    b.step(64)
    for i in frozen:                     # 64 + 64 steps in all, as if never stopped
        assert b.lattice_steps(i) == 128
        assert np.array_equal(b.populations(i), single_run(lbm, descs[i], rhos[i], 128)), i
    # no active lattice: stepping is a no-op
    b.set_active(np.zeros(len(descs), dtype=bool))
    before = [b.populations(i) for i in range(len(descs))]
    b.step(70)
    b.sync()
    for i in range(len(descs)):
        assert np.array_equal(b.populations(i), before[i])
    assert not b.errors().any()
    b.close()
