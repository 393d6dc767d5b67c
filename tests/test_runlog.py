"""The chunked-run log (host logic, CPU): chunking, the record fields, the mass drift
relative to the first record and the JSON-lines file, with a stand-in lattice whose
methods record the calls (the lattice calls themselves are tested on the GPU)."""
import json

import pytest

from paper_1306_6445_gb300.runlog import run_logged


class FakeLattice:
    def __init__(self):
        self.nx, self.ny = 10, 20
        self.steps_done = 0
        self.calls = []

    def sync(self):
        self.calls.append("sync")

    def step(self, n):
        self.calls.append(("step", n))
        self.steps_done += n

    def reduce(self):
        # mass grows by 1e-6 per step, max|v| by 1e-3
        return [1000.0 * (1 + 1e-9 * self.steps_done), 0.0, 0.0, 1e-3 * self.steps_done]

    def measure_droplet(self, radius):
        self.calls.append(("measure", radius))
        return {"theta": 0.01, "rho_in": 0.3, "rho_out": 0.02, "R": radius, "p_in": 0.0,
                "p_out": 0.0, "mass": 0.0, "failed": 0.0}


def test_chunks_records_and_file(tmp_path):
    lat = FakeLattice()
    ticks = iter(range(100))
    path = tmp_path / "run.jsonl"
    recs = run_logged(lat, 25, 10, str(path), radius=12.0, clock=lambda: next(ticks) * 0.5)
    assert [c[1] for c in lat.calls if isinstance(c, tuple) and c[0] == "step"] == [10, 10, 5]
    assert [r["step"] for r in recs] == [10, 20, 25]
    assert recs[0]["mass_drift"] == 0.0
    assert recs[2]["mass_drift"] == pytest.approx((1 + 25e-9) / (1 + 10e-9) - 1, rel=1e-9)
    assert recs[1]["max_v"] == pytest.approx(0.02)
    # 0.5 s per chunk on the fake clock
    assert recs[0]["mlups"] == pytest.approx(10 * 20 * 10 / 0.5 / 1e6)
    assert recs[2]["theta"] == 0.01 and recs[2]["rho_in"] == 0.3
    lines = [json.loads(s) for s in path.read_text().splitlines()]
    assert lines == recs


def test_no_droplet_fields_without_a_radius_and_argument_checks(tmp_path):
    lat = FakeLattice()
    recs = run_logged(lat, 3, 5, str(tmp_path / "a.jsonl"))
    assert len(recs) == 1 and "theta" not in recs[0]
    assert run_logged(lat, 0, 5, str(tmp_path / "b.jsonl")) == []
    with pytest.raises(ValueError):
        run_logged(lat, 5, 0, str(tmp_path / "c.jsonl"))
