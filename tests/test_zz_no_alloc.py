"""lb_reduce_noalloc, the reduction entry point for callers that cannot allocate device
memory (for example code confined to a device-memory budget given to it by its host
application, or code that must not call cudaMalloc/cudaFree because they can synchronise
the device). Its scratch is a static device array instead of an allocation, so this test
checks that it returns what lb_reduce returns, on two calls in a row (the second call
must not be disturbed by what the first left in the shared array).

The file name makes pytest collect it last."""
import numpy as np
import pytest

from paper_1306_6445_gb300 import inputs as I

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


def close(a, ref, mass):
    # the tolerance of the reduction parity test: 1e-13 relative to the total mass
    assert a[0] == pytest.approx(ref[0], rel=1e-13)
    assert abs(a[1] - ref[1]) <= 1e-13 * mass
    assert abs(a[2] - ref[2]) <= 1e-13 * mass
    assert a[3] == pytest.approx(ref[3], rel=1e-13)


@pytest.mark.parametrize("prec,walls,nx,ny", [("fp64", True, 96, 70), ("fp32", False, 512, 384),
                                              ("fp64", False, 2048, 2048)])
def test_noalloc_reduction_matches_lb_reduce_twice(lbm, prec, walls, nx, ny):
    eos = lbm.cs_eos(0.8)
    rates = lbm.RateParams.from_viscosity(0.1)
    rho = I.droplet_density(nx, ny, min(nx, ny) / 5.0, 0.31, 0.02)
    ux, uy = I.random_velocity(np.random.default_rng(3), rho.shape, 0.01)
    lat = lbm.Lattice(nx, ny, eos, -1.0, kappa=0.3, rates=rates, prec=prec, walls_y=walls)
    lat.set_rho_u(rho, ux, uy)
    lat.step(25)
    ref = lat.reduce()
    first = lbm.lb_reduce_noalloc(lat.ctx)
    second = lbm.lb_reduce_noalloc(lat.ctx)
    close(first, ref, ref[0])
    close(second, ref, ref[0])
    # after more steps the shared scratch holds the previous call's values: still exact
    lat.step(5)
    ref2 = lat.reduce()
    close(lbm.lb_reduce_noalloc(lat.ctx), ref2, ref2[0])
    lat.close()


def test_noalloc_reduction_rejects_oversized_lattice(lbm):
    eos = lbm.EOSParams(kind="exp")
    lat = lbm.Lattice(4100, 4100, eos, -40.0, prec="fp32")   # 16.8 M sites > 2^24
    with pytest.raises(lbm.LBError) as ei:
        lbm.lb_reduce_noalloc(lat.ctx)
    assert ei.value.status == lbm.LB_EINVAL
    assert "at most" in str(ei.value)
    lat.close()


def _feq_rest(rho):
    """Populations at rest, f_a = w_a rho (host layout [a][y][x])."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    return w[:, None, None] * rho[None, :, :]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_reports_a_domain_error_like_lb_reduce(lbm, prec):
    """A state with a few sites above the Carnahan-Starling psi^2 > 0 branch (rho > 0.47 at
    0.8 T_c): after one queued step both reductions return LB_EDOMAIN and leave their
    context poisoned."""
    eos = lbm.cs_eos(0.8)
    rho = np.full((40, 48), 0.05)
    rho[20, 10:13] = 0.6
    got = []
    for which in ("lb_reduce", "noalloc"):
        lat = lbm.Lattice(48, 40, eos, -1.0, prec=prec)
        lat.set_populations(_feq_rest(rho))
        lat.step(1)
        with pytest.raises(lbm.LBError) as ei:
            lat.reduce() if which == "lb_reduce" else lbm.lb_reduce_noalloc(lat.ctx)
        got.append((ei.value.status, lbm.lb_status_of(lat.ctx)))
        lat.close()
    assert got[0] == got[1] == (lbm.LB_EDOMAIN, lbm.LB_EDOMAIN)


def test_noalloc_reports_an_earlier_timeout(lbm):
    """A step queued before the call whose bounded wait gave up (the test hook leaves one
    ring row unrequested, so the wait runs out after about a second): lb_reduce_noalloc
    returns LB_ETIMEOUT, as lb_reduce does, and the context stays poisoned."""
    eos = lbm.EOSParams(kind="exp")
    rho = I.droplet_density(64, 64, 12.0, 400.0, 150.0)
    lat = lbm.Lattice(64, 64, eos, -40.0, prec="fp32")
    lat.set_rho_u(rho)
    lbm.lb_debug_stall_row(lat.ctx, 20)
    lat.step(1)
    with pytest.raises(lbm.LBError) as ei:
        lbm.lb_reduce_noalloc(lat.ctx)
    assert ei.value.status == lbm.LB_ETIMEOUT
    assert lbm.lb_status_of(lat.ctx) == lbm.LB_ETIMEOUT
    with pytest.raises(lbm.LBError) as ei:
        lbm.lb_reduce_noalloc(lat.ctx)
    assert ei.value.status == lbm.LB_ETIMEOUT
    lat.close()


@pytest.mark.parametrize("kind", ["bf16", "open"])
def test_noalloc_rejects_bf16_and_open_boundaries(lbm, kind):
    eos = lbm.cs_eos(0.8)
    if kind == "bf16":
        lat = lbm.Lattice(32, 32, eos, -1.0, prec="bf16", storage_shift=0.02)
    else:
        lat = lbm.Lattice(32, 32, eos, -1.0, prec="fp32", open_bc=True)
    lat.set_rho_u(np.full((32, 32), 0.05))
    with pytest.raises(lbm.LBError) as ei:
        lbm.lb_reduce_noalloc(lat.ctx)
    assert ei.value.status == lbm.LB_EINVAL
    # a rejected call does not poison the context
    assert lbm.lb_status_of(lat.ctx) == lbm.LB_OK
    assert lat.reduce()[0] == pytest.approx(0.05 * 32 * 32, rel=1e-2)   # BF16 storage: 8 bits
    lat.close()
