"""The FP64 FMA-rate probe that gives the FP64 update its ALU roof: argument checks, a
rate that does not depend on the loop length (the launch is long enough to time), and a
rate that the FP64 step kernel cannot beat by more than the probe's own timing noise."""
import pytest

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


def test_probe_rejects_bad_arguments(lbm):
    with pytest.raises(lbm.LBError) as e:
        lbm.lb_probe_fp64_fma_rate(None, 0)
    assert e.value.status == lbm.LB_EINVAL


def test_probe_rate_is_independent_of_the_loop_length(lbm):
    r1 = lbm.lb_probe_fp64_fma_rate(None, 2048)
    r2 = lbm.lb_probe_fp64_fma_rate(None, 8192)
    print(f"FP64 FMA rate: {r1 / 1e9:.1f} and {r2 / 1e9:.1f} G/s")
    assert r1 > 0 and r2 > 0
    assert r2 == pytest.approx(r1, rel=0.2)
