"""The JSON-lines observable log (``trace.run_logged``), driven by a stub
solver on the CPU: observation cadence, fields, and stop on divergence."""
import json

from paper_1411_2181_gb300 import trace


class Stub:
    def __init__(self, diverge_at=None):
        self.t = 0
        self.diverge_at = diverge_at

    def step(self, n):
        self.t += n

    def observables(self, k=0, raise_on_diverged=True):
        bad = self.diverge_at is not None and self.t >= self.diverge_at
        return dict(step=self.t, t_over_tem=self.t / 100.0, D=0.01 * self.t, theta_deg=45.0, Lp_over_2R=1.0,
                    necks=0, broken=0, mass=(1.0, 2.0), volume=1.0, flags=1 if bad else 0)


def test_cadence_and_fields(tmp_path):
    path = str(tmp_path / "run.jsonl")
    rows = trace.run_logged(Stub(), 0, steps=25, every=10, path=path)
    assert [r["step"] for r in rows] == [0, 10, 20, 25]
    lines = [json.loads(x) for x in open(path)]
    assert lines == rows
    assert set(lines[0]) == {"instance", *trace.FIELDS} and lines[0]["mass"] == [1.0, 2.0]


def test_stops_at_divergence(tmp_path):
    rows = trace.run_logged(Stub(diverge_at=20), 0, steps=100, every=10, path=str(tmp_path / "d.jsonl"))
    assert [r["step"] for r in rows] == [0, 10, 20]
