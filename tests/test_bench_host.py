"""Host-side helpers of bench.py (CPU): the clock summary taken from nvidia-smi lines, the
lookup of figures in a committed ncu summary (used only while its kernel-source hash is
current), the workload description both arms print and the splash grid's reruns."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test",
                                                  os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_clock_summary(bench):
    c = bench.ClockSampler(0)
    assert c.summary()["reasons"] == ["unsampled"]
    c.samples = [["2070", "2070", "900.1", "Not Active", "Not Active", "Not Active", "Active"],
                 ["1980", "2070", "1390.0", "Not Active", "Not Active", "Not Active", "Active"],
                 ["2070", "2070", "1000.0", "Not Active", "Not Active", "Not Active",
                  "Not Active"],
                 ["[N/A]", "2070", "0", "Not Active", "Active", "Not Active", "Not Active"]]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_profiled_value_only_for_the_current_kernel_source(bench, tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k.md").write_text(
        "# title\n\nkernel_source_sha: abc123\nfigure_x: 42.5\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda prec="fp32": "abc123")
    assert bench.profiled_value("k", "figure_x", "fp32") == 42.5
    assert bench.profiled_value("k", "missing_key", "fp32") is None
    assert bench.profiled_value("absent", "figure_x", "fp32") is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda prec="fp32": "def456")
    assert bench.profiled_value("k", "figure_x", "fp32") is None


def test_kernel_source_hash_is_per_precision_and_stable(bench):
    a, b = bench.kernel_source_sha("fp32"), bench.kernel_source_sha("fp64")
    assert a != b and len(a) == 16
    assert bench.kernel_source_sha("fp32") == a


def test_both_arms_describe_the_same_workload(bench):
    c = bench.bench_config(2048, 2048, 100, 4)
    assert c["workload"] == bench.WORKLOAD and c["parallelism"] == "replicas4"
    assert c["nx"] == c["ny"] == 2048 and c["lb_steps_per_step"] == 100


def test_splash_points_that_break_early_run_again_warmer(bench, monkeypatch):
    """The splash grid reruns, at the warmer temperature, exactly the points that left the
    EOS branch before t* = 1.75 (4000 steps at D = 400, U = 0.05 from t* = 0.05 is
    t* = 0.55; 28000 steps is t* = 3.55), and lists both runs of such a point."""
    calls = []

    def fake_point(lbm, torch, net, nx, ny, D, We, Re, U, t_over_tc, steps):
        calls.append((We, Re, t_over_tc))
        early = We == 800.0 and t_over_tc == 0.65
        late = We == 200.0 and Re == 1000.0
        done = 4000 if early else (28000 if late else steps)
        return {"We": We, "Re": Re, "t_over_tc": t_over_tc, "steps_done": done,
                "breakdown": "LB_EDOMAIN" if (early or late) else None}

    monkeypatch.setattr(bench, "splash_point", fake_point)
    out = bench.splash_leg(None, None, None, steps=40000)
    assert calls == [(200.0, 500.0, 0.65), (200.0, 1000.0, 0.65),
                     (800.0, 500.0, 0.65), (800.0, 500.0, 0.70),
                     (800.0, 1000.0, 0.65), (800.0, 1000.0, 0.70)]
    assert [(p["We"], p["Re"], p["t_over_tc"]) for p in out["points"]] == calls
    assert "0.7Tc" in out["workload"]
