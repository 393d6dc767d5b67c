"""GPU diagnostics of single lattices (the every-k-steps reductions next to the update):
the Laplace measurement of a droplet (lb_measure_droplet) against the same sums recomputed
on the host from the GPU's own density field with the oracle's bulk pressure, and against
the batched measurement of the same state (an independent GPU path with another
summation order); the interface height per column (lb_interface_height) against the
oracle's interface height on every column of the same density field, bit for bit,
including the columns and thresholds that have no interface."""
import numpy as np
import pytest

from oracle import diagnostics as D
from oracle import lattice as OL
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


def host_laplace(rho, params, radius):
    """The measurement's definitions written out on the host (masks from the given radius)."""
    ny, nx = rho.shape
    pres = OL.pressure(rho, params)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    r = np.hypot(x - (nx - 1) / 2, y - (ny - 1) / 2)
    inside = r < radius / 2
    outside = r > radius + 0.3 * min(nx, ny) / 2
    rho_in, rho_out = rho[inside].mean(), rho[outside].mean()
    p_in, p_out = pres[inside].mean(), pres[outside].mean()
    R = np.sqrt((rho.sum() - rho_out * rho.size) / (np.pi * (rho_in - rho_out)))
    return {"theta": (p_in - p_out) * R, "rho_in": rho_in, "rho_out": rho_out, "R": R,
            "p_in": p_in, "p_out": p_out, "mass": rho.sum()}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["cs", "exp"])
def test_droplet_measurement_matches_host_sums(lbm, prec, kind):
    if kind == "cs":
        eos, G = lbm.cs_eos(0.8), -1.0
        rv, rl, _ = lbm.lb_maxwell(eos, G)
    else:                                         # Sec. V.A: psi0 = 4, rho0 = 200, G = -40
        eos, G = lbm.EOSParams(kind="exp"), -40.0
        rv, rl, _ = lbm.lb_maxwell(eos, G)
    rates = lbm.RateParams.from_viscosity(0.1)
    nx, ny, R = 301, 203, 45.0                    # ragged in both directions
    lat = lbm.Lattice(nx, ny, eos, G, kappa=0.5, rates=rates, prec=prec)
    lat.set_rho_u(I.droplet_density(nx, ny, R, rl, rv))
    lat.step(400)
    m = lat.measure_droplet(R)
    again = lat.measure_droplet(R)
    rho = lat.rho()
    mass = lat.reduce()[0]
    lat.close()
    ref = host_laplace(rho, oracle_params(eos, G, 0.5, 0.0, rates), R)
    assert again == m                              # fixed summation order
    assert m["failed"] == 0
    # densities are the GPU's own (FP64 sums in another order); the pressure is computed
    # in the lattice's arithmetic on the GPU and in FP64 by the oracle
    assert m["rho_in"] == pytest.approx(ref["rho_in"], rel=1e-12)
    assert m["rho_out"] == pytest.approx(ref["rho_out"], rel=1e-12)
    assert m["mass"] == pytest.approx(ref["mass"], rel=1e-12)
    assert m["mass"] == pytest.approx(mass, rel=1e-12)
    assert m["R"] == pytest.approx(ref["R"], rel=1e-10)
    # p = rho/3 + (G/2) psi^2 is a small difference of two terms of size about rho_in/3:
    # bound its error by the size of the terms (FP32 psi: a few units of 6e-8 relative)
    scale = ref["rho_in"] / 3.0
    p_abs = 1e-13 * scale if prec == "fp64" else 4e-6 * scale
    assert abs(m["p_in"] - ref["p_in"]) <= p_abs
    assert abs(m["p_out"] - ref["p_out"]) <= p_abs
    assert abs(m["theta"] - ref["theta"]) <= 2.0 * p_abs * ref["R"] + 1e-12 * abs(ref["theta"])


def test_droplet_measurement_equals_the_batched_measurement(lbm):
    eos = lbm.cs_eos(0.75)
    rv, rl, _ = lbm.lb_maxwell(eos, -1.0)
    rates = lbm.RateParams.from_viscosity(0.15)
    nx, ny, R = 160, 130, 30.0
    rho0 = I.droplet_density(nx, ny, R, rl, rv)
    lat = lbm.Lattice(nx, ny, eos, -1.0, kappa=0.3, sigma_force=0.087, rates=rates, prec="fp64")
    lat.set_rho_u(rho0)
    lat.step(500)
    m = lat.measure_droplet(R)
    f = lat.populations()
    lat.close()
    b = lbm.Batch([lbm.LatticeDesc(nx, ny, eos, -1.0, kappa=0.3, sigma_force=0.087, rates=rates)],
                  prec="fp64")
    b.set_rho_u(0, rho0)
    b.step(500)
    assert np.array_equal(b.populations(0), f)    # the same state
    mb = b.measure(np.array([R]))[0]
    b.close()
    for k, key in enumerate(("theta", "rho_in", "rho_out", "R", "p_in", "p_out", "mass")):
        assert m[key] == pytest.approx(mb[k], rel=1e-9 if key == "theta" else 1e-12), key
    assert mb[7] == 0 and m["failed"] == 0


def test_droplet_measurement_argument_errors(lbm):
    eos = lbm.cs_eos(0.8)
    lat = lbm.Lattice(64, 64, eos, -1.0, prec="fp32")
    rv, rl, _ = lbm.lb_maxwell(eos, -1.0)
    lat.set_rho_u(I.droplet_density(64, 64, 12.0, rl, rv))
    for bad in (0.0, -3.0, float("nan"), float("inf")):
        with pytest.raises(lbm.LBError) as e:
            lat.measure_droplet(bad)
        assert e.value.status == lbm.LB_EINVAL
    with pytest.raises(lbm.LBError) as e:
        lat.interface_height(float("nan"))
    assert e.value.status == lbm.LB_EINVAL
    lat.step(1)                                    # the context is still usable
    lat.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("bc", ["walls", "open"])
def test_interface_height_equals_the_oracle_on_the_same_field(lbm, prec, bc):
    if prec == "bf16" and bc == "open":
        pytest.skip("open boundaries are not compiled for BF16 storage")
    eos = lbm.cs_eos(0.8)
    rv, rl, _ = lbm.lb_maxwell(eos, -1.0)
    rates = lbm.RateParams.from_viscosity(0.1)
    nx, ny = 301, 131                              # ragged strips and row segments
    rho0 = I.layer_density(nx, ny, 50.0, rl, rv, amplitude=6.0, wavenumber=2)
    kw = {"walls_y": True} if bc == "walls" else {"open_bc": True}
    lat = lbm.Lattice(nx, ny, eos, -1.0, kappa=0.4, rates=rates, prec=prec,
                      storage_shift=rv, **kw)
    lat.set_rho_u(rho0)
    lat.step(200)
    rho = lat.rho()
    mid = 0.5 * (rl + rv)
    # a threshold inside the interface, one above every density (row 0 is already below:
    # NaN) and one below every density (no row is below: NaN)
    for thr in (mid, 2.0 * rho.max(), 0.5 * rho.min()):
        got = lat.interface_height(thr)
        ref = np.array([D.interface_height(rho[:, x], thr) for x in range(nx)])
        assert np.array_equal(got, ref, equal_nan=True), thr
    h = lat.interface_height(mid)
    lat.close()
    assert np.all(np.isfinite(h)) and abs(np.nanmean(h) - 50.0) < 3.0


def test_run_log_records_match_the_library_calls(lbm, tmp_path):
    from paper_1306_6445_gb300.runlog import run_logged

    eos = lbm.cs_eos(0.8)
    rv, rl, _ = lbm.lb_maxwell(eos, -1.0)
    lat = lbm.Lattice(64, 64, eos, -1.0, kappa=0.3, rates=lbm.RateParams.from_viscosity(0.1),
                      prec="fp32")
    lat.set_rho_u(I.droplet_density(64, 64, 16.0, rl, rv))
    recs = run_logged(lat, 30, 10, str(tmp_path / "run.jsonl"), radius=16.0)
    m = lat.measure_droplet(16.0)
    red = lat.reduce()
    lat.close()
    assert [r["step"] for r in recs] == [10, 20, 30]
    assert recs[-1]["theta"] == m["theta"] and recs[-1]["rho_in"] == m["rho_in"]
    assert recs[-1]["mass"] == red[0] and recs[-1]["max_v"] == red[3]
    assert abs(recs[-1]["mass_drift"]) < 1e-5 and all(r["mlups"] > 0 for r in recs)
