"""The study's break-up details and the time-series runner on the GPU, on
cases far from any threshold at the study's resolution (W = 40): a
matrix-viscoelastic droplet at Ca = 2.0 (its Ca_cr is about 1.1 at
2R/W = 0.6) breaks, a Newtonian droplet at Ca = 0.8 (Ca_cr about 2.1)
stays whole."""
import json
import os

import pytest

from paper_1411_2181_gb300 import study

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    from paper_1411_2181_gb300 import build
    build.build()


def test_breakup_details(built):
    cases = [study.Case(Ca=2.0, De=2.0, lam=1.0, conf=0.6, phase=2, seed=7),
             study.Case(Ca=0.8, De=0.0, lam=1.0, conf=0.6, phase=1, seed=7)]
    broke, whole = study.breakup_details(cases, every_tem=0.5, after_tem=1.0)
    assert broke["ok"] and whole["ok"]
    assert broke["t_break"] is not None and 0 < broke["t_break"] <= study.T_MAX_TEM + 0.5
    assert broke["fragments_at_break"] >= 2 and broke["fragments_after"][0] == broke["fragments_at_break"]
    assert broke["fragments_max"] == max(broke["fragments_after"]) and len(broke["fragments_after"]) >= 2
    assert whole["t_break"] is None and whole["fragments_after"] == [] and whole["fragments_max"] == 0


def test_time_series_runner(built, tmp_path):
    from paper_1411_2181_gb300 import trace
    out = os.path.join(tmp_path, "ts.jsonl")
    trace.main(["--ca", "0.2", "--steps", "400", "--every", "200", "--out", out])
    rows = [json.loads(line) for line in open(out)]
    assert [r["step"] for r in rows] == [0, 200, 400]
    assert all(r["Ca"] == 0.2 and set(trace.FIELDS) <= set(r) for r in rows)
    assert rows[-1]["D"] > rows[0]["D"] and not os.path.exists(out + ".part")
