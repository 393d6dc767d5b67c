"""The κ-choice logic of the surrogate's check and fallback (`surrogate.tune_kappa`), on the
CPU. The Laplace runs are replaced by a synthetic surface tension
sigma(T, kappa) = sigma_0(T) (1 - kappa)^p, whose exponent p != 1 stands for the departure
from the leading-order law of Eq. 22 that the paper's Table 2 shows at large kappa. The
network is a stand-in with a known answer (or none). This checks the bookkeeping:
one run per target when the network is right; the law, then the secant in
ln sigma against ln(1 - kappa), otherwise; and failed runs."""
import numpy as np
import pytest

from paper_1306_6445_gb300 import surrogate, sweep


P_EXP = 1.15


def sigma0(t):
    return 0.01 * (1.0 - np.asarray(t)) ** 1.5


def fake_sigma(t, kappa):
    return sigma0(t) * (1.0 - np.asarray(kappa)) ** P_EXP


class FakeNet:
    """invert_kappa returns the exact kappa scaled by `bias` (NaN where `nan_mask`)."""

    def __init__(self, bias=1.0, nan_mask=None):
        self.bias, self.nan_mask = bias, nan_mask

    def invert_kappa(self, q, lo, hi):
        t, s = q[:, 0], q[:, 2]
        k = 1.0 - (s / sigma0(t)) ** (1.0 / P_EXP)
        k = np.clip(k * self.bias, lo, hi)
        if self.nan_mask is not None:
            k = np.where(self.nan_mask, np.nan, k)
        return k.astype(np.float32)


@pytest.fixture
def runs_log(monkeypatch):
    calls = []

    def fake_points(lbm, t, kappa, tau, **kw):
        calls.append(len(t))
        return fake_sigma(t, kappa)

    monkeypatch.setattr(surrogate, "sweep_points", fake_points)
    return calls


def targets():
    t = np.array([0.7, 0.8, 0.9, 0.8])
    kappa_true = np.array([0.3, 0.6, 0.85, 0.93])
    return t, np.full(4, 0.8), fake_sigma(t, kappa_true), kappa_true


def test_a_right_network_needs_one_run_per_target(runs_log):
    t, tau, s, k = targets()
    r = surrogate.tune_kappa(None, FakeNet(), t, tau, s, tol=0.02)
    assert np.all(r["runs"] == 1) and runs_log == [4]
    assert np.allclose(r["kappa"], k, atol=1e-5)
    assert np.all(np.abs(r["rel_err"]) < 1e-4)


def test_without_a_network_the_law_then_the_secant_reach_the_target(runs_log):
    t, tau, s, k = targets()
    r = surrogate.tune_kappa(None, None, t, tau, s, tol=0.005, max_rounds=4)
    assert np.all(np.abs(r["rel_err"]) <= 0.005)
    # a kappa = 0 run, the law's kappa, then secant steps: at least 2 runs each, and
    # the first batched run measured all four at kappa = 0
    assert np.all(r["runs"] >= 2) and runs_log[0] == 4
    assert np.allclose(r["kappa"], k, atol=5e-3)


def test_a_biased_network_is_caught_by_the_check_and_corrected(runs_log):
    t, tau, s, k = targets()
    r = surrogate.tune_kappa(None, FakeNet(bias=0.9), t, tau, s, tol=0.01)
    assert np.all(np.abs(r["rel_err"]) <= 0.01)
    assert np.all(r["runs"] >= 2)                  # each first try missed by > 1 %


def test_targets_outside_the_network_go_straight_to_the_fallback(runs_log):
    t, tau, s, k = targets()
    net = FakeNet(nan_mask=np.array([False, True, False, False]))
    r = surrogate.tune_kappa(None, net, t, tau, s, tol=0.02)
    assert runs_log[0] == 3                       # the NaN target was not run at NaN
    assert r["runs"][1] >= 2 and np.all(r["runs"][[0, 2, 3]] == 1)
    assert np.all(np.abs(r["rel_err"]) <= 0.02)


def test_failed_runs_stay_failed_and_are_reported(monkeypatch):
    def failing(lbm, t, kappa, tau, **kw):
        return np.full(len(t), np.nan)

    monkeypatch.setattr(surrogate, "sweep_points", failing)
    t, tau, s, k = targets()
    r = surrogate.tune_kappa(None, FakeNet(), t, tau, s, tol=0.02, max_rounds=2)
    assert np.all(np.isnan(r["sigma"])) and np.all(np.isnan(r["rel_err"]))


# ---- the converged sweep protocol (sweep.converged_readings) against a fake batch ------

class FakeBatch:
    """Stands in for lbm.Batch: lattice i reads theta_i(t) = target_i (1 + a_i cos(t / p_i)
    exp(-t / tau_i) + d_i exp(-t / tau_d)); set_active must come at even step counts, like
    the library's."""

    def __init__(self, target, amp, tau, period=None, drift=None, tau_d=3000.0):
        self.target, self.amp, self.tau = map(np.asarray, (target, amp, tau))
        self.n = len(self.target)
        self.period = np.full(self.n, 50.0) if period is None else np.asarray(period)
        self.drift = np.zeros(self.n) if drift is None else np.asarray(drift)
        self.tau_d = tau_d
        self.t = np.zeros(self.n)
        self.active = np.ones(self.n, dtype=bool)
        self.steps = 0
        self.calls = []

    def step(self, k):
        assert k > 0
        self.t[self.active] += k
        self.steps += k

    def measure(self, radii):
        th = self.target * (1 + self.amp * np.cos(self.t / self.period) * np.exp(-self.t / self.tau)
                            + self.drift * np.exp(-self.t / self.tau_d))
        out = np.zeros((self.n, 8))
        out[:, 0], out[:, 1], out[:, 2] = th, 0.3, 0.02
        return out

    def set_active(self, active):
        assert self.steps % 2 == 0
        self.active = np.asarray(active, dtype=bool).copy()
        self.calls.append((self.steps, self.active.copy()))


def test_step_budget_grows_with_the_square_of_the_side():
    assert sweep.step_budget(64) == 8192                    # the floor
    assert sweep.step_budget(512) == 131072                 # 0.5 * 512^2
    assert sweep.step_budget(384) % sweep.WINDOW == 0 and sweep.step_budget(384) >= 73728


def test_converged_readings_retires_each_lattice_at_its_budget():
    budgets = np.array([8192, 16384, 8192, 32768])
    b = FakeBatch(target=[1e-3, 2e-3, 3e-3, 4e-3], amp=[0.5, 0.5, 0.5, 0.5],
                  tau=[500.0, 500.0, 1e9, 500.0])
    r = sweep.converged_readings(b, budgets, np.ones(4), extensions=0)
    # every lattice took exactly its budget and the batch stopped with the last one
    assert np.array_equal(b.t, budgets) and b.steps == budgets.max()
    assert np.array_equal(r["steps"], budgets)
    # retirements at the budgets, in order
    assert [c[0] for c in b.calls] == [8192, 16384, 32768]
    # damped lattices read their target; the undamped one (tau = inf) oscillates between
    # windows and is not converged
    ok = [0, 1, 3]
    assert np.allclose(r["theta"][ok], b.target[ok], rtol=1e-6)
    assert r["converged"][ok].all() and not r["converged"][2]
    # the reading is the mean over the last window (32 readings of the fake's curve)
    ts = np.arange(8192 - 2048 + 64, 8192 + 1, 64)
    want = np.mean(3e-3 * (1 + 0.5 * np.cos(ts / 50.0) * np.exp(-ts / 1e9)))
    assert r["theta"][2] == pytest.approx(want, rel=1e-12)
    # the check reading: the window before 3/4 of the budget
    tc = np.arange(6144 - 2048 + 64, 6144 + 1, 64)
    assert r["theta_check"][2] == pytest.approx(
        np.mean(3e-3 * (1 + 0.5 * np.cos(tc / 50.0) * np.exp(-tc / 1e9))), rel=1e-12)


def test_converged_readings_runs_slow_lattices_on():
    # lattice 1 still drifts at its budget (exp(-t/3000)): it runs on for half its budget at
    # a time until two readings agree (3 % apart at 6144/8192 steps, 2.4 % at 8192/12288,
    # 0.6 % at 12288/16384); lattice 0 converges at once; lattice 2 swings slowly (a period
    # of 12 600 steps, undamped) and stops unconverged after the allowed extensions
    budgets = np.array([8192, 8192, 8192])
    b = FakeBatch(target=[1e-3, 1e-3, 1e-3], amp=[0.5, 0.0, 0.3], tau=[300.0, 1.0, 1e12],
                  period=[50.0, 50.0, 2000.0], drift=[0.0, 0.5, 0.0])
    r = sweep.converged_readings(b, budgets, np.ones(3), extensions=2)
    assert r["steps"][0] == 8192 and r["converged"][0]
    assert r["steps"][1] == 16384 and r["converged"][1]
    assert r["steps"][2] == 8192 + 2 * 4096 and not r["converged"][2]
    assert np.array_equal(b.t, r["steps"])
    assert r["theta"][1] == pytest.approx(1e-3, rel=0.005)   # the drift left: 0.3 %
    # the batch was told each time a lattice stopped, at the step it stopped
    assert [c[0] for c in b.calls] == [8192, 16384]


def test_converged_readings_rejects_budgets_off_the_window():
    b = FakeBatch([1.0], [0.0], [1.0])
    with pytest.raises(ValueError):
        sweep.converged_readings(b, [5000], [1.0])
    with pytest.raises(ValueError):
        sweep.converged_readings(b, [4096], [1.0])   # fewer than four windows
