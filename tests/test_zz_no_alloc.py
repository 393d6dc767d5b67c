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
