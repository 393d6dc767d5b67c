"""The C-ABI library loads and exports every function include/*.h declares; host-only
helpers (no GPU work) agree with the oracle's thermodynamics. CPU only."""
import ctypes
import os
import re

import pytest

from oracle import eos as OE

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbm():
    from paper_1306_6445_gb300 import _build

    _build.build()
    from paper_1306_6445_gb300 import lbm as mod

    mod.load_library()
    return mod


def header_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^[\w \*]*?\b(lb_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_header_declares_the_documented_entry_points():
    names = header_functions()
    for need in ("lb_init", "lb_step", "lb_get_rho", "lb_get_u", "lb_reduce", "lb_free",
                 "lb_mlp_train", "lb_mlp_forward", "lb_mlp_loss_grad", "lb_mlp_invert_kappa"):
        assert need in names


def test_library_exports_every_declared_symbol(lbm):
    lib = ctypes.CDLL(lbm.LIB_PATH)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps exactly the declared set
    assert sorted(lbm.EXPORTED) == header_functions()


def test_pitch_and_buffer_size(lbm):
    # nx + 2 H elements (H = 8 for FP32, 4 otherwise), rounded up to 32 elements
    assert lbm.lb_pitch(1, lbm.LB_FP32) == 32
    assert lbm.lb_pitch(2033, lbm.LB_FP32) == 2080
    assert lbm.lb_pitch(2033, lbm.LB_FP64) == 2048
    assert lbm.lb_pitch(2033, lbm.LB_BF16) == 2048
    assert lbm.lb_pitch(2048, lbm.LB_FP64) == 2080
    assert lbm.lb_pitch(2024, lbm.LB_FP32) == 2048
    assert lbm.lb_buffer_bytes(100, 7, lbm.LB_FP64) == 9 * 7 * 128 * 8
    assert lbm.lb_buffer_bytes(0, 7, lbm.LB_FP64) == 0


def test_cs_critical_point_agrees_with_oracle(lbm):
    Tc, rc = lbm.lb_cs_critical(1.0, 4.0, 1.0)
    oTc, orc = OE.cs_critical(1.0, 4.0, 1.0)
    assert Tc == pytest.approx(oTc, rel=1e-9)
    assert rc == pytest.approx(orc, rel=1e-5)   # flat maximum: rho_c is less sharp than T_c


@pytest.mark.parametrize("case", ["cs0.7", "cs0.8", "cs0.9", "exp", "piecewise"])
def test_maxwell_host_helper_agrees_with_oracle(lbm, case):
    if case.startswith("cs"):
        t = float(case[2:])
        eos, G = lbm.cs_eos(t), -1.0
        oeos = OE.EOS(kind="cs", T=eos.T)
    elif case == "exp":
        eos, G, oeos = lbm.EOSParams(kind="exp"), -40.0, OE.EOS(kind="exp")
    else:
        eos, G, oeos = lbm.EOSParams(kind="piecewise"), -1.0, OE.colosqui_eos()
    rv, rl, pb = lbm.lb_maxwell(eos, G)
    orv, orl, opb = OE.maxwell(oeos, G)
    assert rv == pytest.approx(orv, rel=1e-7)
    assert rl == pytest.approx(orl, rel=1e-7)


def test_init_rejects_bad_arguments_without_touching_the_gpu(lbm):
    eos = lbm.EOSParams(kind="exp")
    good = lbm.RateParams()
    bad_cases = [
        dict(nx=2, ny=8),                                   # too small
        dict(rates=lbm.RateParams(s_v=2.0)),                # tau = 1/2
        dict(rates=lbm.RateParams(s_e=0.0)),
        dict(kappa=1.0),                                    # kappa outside [0, 1)
        dict(kappa=-0.1),
        dict(sigma=0.1, rates=lbm.RateParams(s_e=0.8, s_zeta=1.0)),   # Eq. 8 needs tau_zeta = tau_e
        dict(prec=7),
        dict(eos=lbm.EOSParams(kind="cs", T=0.07), G=0.0),  # EOS-based psi divides by G
    ]
    for kw in bad_cases:
        args = dict(nx=8, ny=8, eos=eos, G=-40.0, kappa=0.0, sigma=0.0, rates=good,
                    prec=lbm.LB_FP64)
        args.update(kw)
        with pytest.raises(lbm.LBError) as ei:
            lbm.lb_init(args["nx"], args["ny"], args["eos"], args["G"], args["kappa"],
                        args["sigma"], args["rates"], args["prec"], lbm.LB_BC_PERIODIC)
        assert ei.value.status == lbm.LB_EINVAL


def test_binding_fails_loudly_without_the_library(lbm, monkeypatch, tmp_path):
    monkeypatch.setattr(lbm, "_lib", None)
    monkeypatch.setattr(lbm, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="CUDA library missing"):
        lbm.load_library()


def test_strip_widths_start_on_16_byte_boundaries(lbm):
    """The batched step's TMA boxes start at each strip's first column, which must be a
    multiple of 4 (16 bytes of FP32): every strip but the last is a whole number of 4-column
    groups, widths fit the kernel's strip and add up to nx."""
    for tx in (64, 128, 240):
        for nx in list(range(1, 700)) + [1021, 2048, 4097]:
            w = lbm.lb_strip_widths(nx, tx)
            assert len(w) == -(-nx // tx)
            assert sum(w) == nx
            assert all(1 <= v <= tx for v in w)
            assert max(w) - min(w) <= 7          # whole 4-column groups; the last may be partial
            starts = [sum(w[:k]) for k in range(len(w))]
            assert all(s % 4 == 0 for s in starts)
    with pytest.raises(lbm.LBError):
        lbm.lb_strip_widths(100, 130)      # strip width not a multiple of 4
