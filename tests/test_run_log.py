"""The JSONL run log of the Python layer (salec.run_logged), on a stand-in simulation with
the read-outs of salec.Sim (no GPU): one line per call of `every` steps with the fields a
run's history needs, and the log stops at the line that shows a failure."""
import json

import numpy as np

from paper_2403_04267_gb300 import salec


class FakeSim:
    def __init__(self, fail_at=None):
        self.n, self.t, self.fail_at = 0, 0.0, fail_at

    def step(self, n):
        self.n += n
        self.t += 0.5 * n

    def scalars(self):
        st = 1 if self.fail_at is not None and self.n >= self.fail_at else 0
        return {"t": self.t, "dt": 0.5, "nstep": self.n, "status": st, "mass_out": 0.0, "mass_discarded": 1.0,
                "mass_pml": 2.0, "zmom_out": 3.0}

    def conservation(self):
        return {"mass": 10.0, "zmom": -1.0, "ke": 2.0, "ie": 3.0}

    def get(self, name):
        assert name == "pmax"
        return np.full((3, 4), 7.0 + self.n)

    def crater(self, z, npts):
        return {"depth": 0.1 * self.n, "diameter": 0.2 * self.n}


def test_run_log_lines(tmp_path):
    path = tmp_path / "run.jsonl"
    recs = salec.run_logged(FakeSim(), 25, 10, str(path), z_surface=0.0)
    lines = [json.loads(l) for l in path.read_text().splitlines()]
    assert lines == recs
    assert [r["step"] for r in recs] == [10, 20, 25]
    assert recs[-1]["t"] == 12.5 and recs[-1]["dt"] == 0.5 and recs[-1]["status"] == 0
    assert recs[0]["sums"] == {"mass": 10.0, "zmom": -1.0, "ke": 2.0, "ie": 3.0}
    assert recs[0]["tallies"]["mass_pml"] == 2.0 and recs[0]["pmax"] == 17.0
    assert recs[-1]["crater"] == {"depth": 2.5, "diameter": 5.0}


def test_run_log_stops_at_a_failure(tmp_path):
    path = tmp_path / "run.jsonl"
    recs = salec.run_logged(FakeSim(fail_at=15), 100, 10, str(path))
    assert [r["step"] for r in recs] == [10, 20]
    assert recs[-1]["status"] == 1 and "crater" not in recs[-1]
