"""Host logic of the Ca_cr searches with a stand-in verdict (no GPU): the
verdict of a case is 'broken' iff Ca exceeds a known threshold that depends
on the triple, so both modes must bracket that threshold within the
tolerance, and the proposal mode must spend fewer runs when its guess is
close."""
import numpy as np
import pytest

from paper_1411_2181_gb300 import study


def fake_threshold(c):
    De, lam, conf, phase = c.De, c.lam, c.conf, c.phase
    return 1.0 + 0.3 * conf + 0.1 * De - 0.2 * (phase == 2) + 0.05 * lam


@pytest.fixture
def fake_runs(monkeypatch):
    calls = []

    def run_batch(cases, device=None, stats=None):
        calls.append(len(cases))
        if stats is not None:
            stats["runs"] = stats.get("runs", 0) + len(cases)
            stats["seconds"] = stats.get("seconds", 0.0)
            stats["lattice_updates"] = 0
        return [study.Verdict(c.Ca > fake_threshold(c), 0.1, 30.0, 0, float("nan")) for c in cases]

    monkeypatch.setattr(study, "run_batch", run_batch)
    return calls


TRIPLES = [(0.0, 1.0, 0.65, 1), (2.0, 0.5, 0.75, 2), (1.0, 1.0, 0.7, 2), (0.5, 0.5, 0.62, 1)]


def test_bisection_brackets_threshold(fake_runs):
    searches, stats = study.search_bisect(TRIPLES, tol=0.02)
    for s in searches:
        th = fake_threshold(study._case(s.triple, 0.0, 0))
        assert s.lo <= th < s.hi and s.width <= 0.02
    # 2 checks + ceil(log2((CA_MAX - CA_MIN) / 0.02)) = 7 halvings per triple
    assert all(s.runs == 9 for s in searches)
    assert stats["rounds"] == 8


class FakeNetwork:
    """A proposal network stand-in whose logit crosses 0 at the threshold
    plus an offset (the network's error)."""

    def __init__(self, offset):
        self.offset = offset

    def forward(self, X):
        ca = X[:, 0] * study.CA_HALF + study.CA_MID
        cases = [study.Case(Ca=0.0, De=float(x[1] + 1.0), lam=float(np.exp(x[2] * np.log(2.0))),
                            conf=float(x[3] * 0.1 + 0.7), phase=1 if x[5] < 0 else 2) for x in X]
        th = np.array([fake_threshold(c) for c in cases]) + self.offset
        y = np.zeros((len(X), 4), np.float32)
        y[:, 2] = (ca - th) * 10
        return y


@pytest.mark.parametrize("offset", [0.0, 0.03, -0.05, 0.2, 5.0, -5.0])
def test_proposal_mode_brackets_threshold(fake_runs, offset):
    searches, stats = study.search_mlp(TRIPLES, FakeNetwork(offset), tol=0.02, delta=0.06)
    for s in searches:
        th = fake_threshold(study._case(s.triple, 0.0, 0))
        assert s.lo <= th < s.hi and s.width <= 0.02
        # the lower end was verified stable and the upper end broken
        lows = [ca for ca, br in s.history if not br]
        highs = [ca for ca, br in s.history if br]
        assert max(lows) == pytest.approx(s.lo) and min(highs) == pytest.approx(s.hi)


def test_proposal_saves_runs_when_close(fake_runs):
    sb, _ = study.search_bisect(TRIPLES, tol=0.02)
    sm, stm = study.search_mlp(TRIPLES, FakeNetwork(0.01), tol=0.02, delta=0.06)
    assert sum(s.runs for s in sm) < sum(s.runs for s in sb)
    for b, m in zip(sb, sm):
        assert abs(0.5 * (b.lo + b.hi) - 0.5 * (m.lo + m.hi)) <= 0.02


def test_features_scaling():
    c = study.Case(Ca=study.CA_MID, De=1.0, lam=1.0, conf=0.7, L2=200.0, phase=1)
    x = study.features([c])[0]
    assert np.allclose(x, [0, 0, 0, 0, 0, -1], atol=1e-6)


def test_range_ends_need_one_run_when_predicted(fake_runs):
    """A network predicting stability over the whole range spends one run to
    confirm it (the threshold lies above the range here)."""
    searches, _ = study.search_mlp(TRIPLES, FakeNetwork(5.0), tol=0.02, delta=0.06, hi=1.0)
    for s in searches:
        assert s.lo == s.hi == 1.0 and s.runs == 1


def test_autotune_candidates():
    """Launch shapes the autotuner tries: every tile height of the one-cell
    kernel, the two-cell kernel only when every Lx is even, and only 8-row
    tiles with the second-order advection scheme; z-chunks no deeper than
    the deepest instance."""
    from dataclasses import replace
    from paper_1411_2181_gb300 import autotune
    from paper_1411_2181_gb300.params import Params
    p = Params(Lx=64, Ly=32, Lz=24)
    shapes = {(k, ty) for k, ty, _ in autotune.candidates([p])}
    assert shapes == {(0, 8), (0, 12), (0, 16), (1, 16)}
    assert all(zc <= 24 for _, _, zc in autotune.candidates([p]))
    odd = {(k, ty) for k, ty, _ in autotune.candidates([p, replace(p, Lx=63)])}
    assert (1, 16) not in odd
    adv = {(k, ty) for k, ty, _ in autotune.candidates([replace(p, advection=1)])}
    assert adv == {(0, 8)}
    assert autotune._key([p], "gpu") != autotune._key([replace(p, advection=1)], "gpu")


def test_training_cases_cover_the_transition():
    """Seven in ten training cases are matrix-viscoelastic with Ca from a
    chosen lower end; the others span the whole range; all lie inside
    [CA_MIN, CA_MAX] with confinements in [CONF_MIN, CONF_MAX]."""
    cs = study.sample_cases(2000, seed=100, mv_ca_from=1.0)
    mv = [c for c in cs if c.phase == 2]
    assert 0.65 < len(mv) / len(cs) < 0.75
    assert all(c.De > 0 for c in mv)
    assert all(1.0 <= c.Ca <= study.CA_MAX for c in mv)
    assert min(c.Ca for c in study.sample_cases(2000, seed=100) if c.phase == 2) < 0.7
    assert all(study.CA_MIN <= c.Ca <= study.CA_MAX and study.CONF_MIN <= c.conf <= study.CONF_MAX for c in cs)


def test_held_out_triples_are_not_training_cases():
    from paper_1411_2181_gb300 import study_run
    tr = study_run.held_out_triples(16)
    assert len(set(tr)) == 16
    assert all(t[3] == 2 and t[0] in (1.0, 1.5, 2.0) for t in tr)
    seen = {(c.De, c.lam, round(c.conf, 6), c.phase) for c in study.sample_cases(2000, seed=100)}
    assert not any((t[0], t[1], round(t[2], 6), t[3]) in seen for t in tr)


@pytest.mark.parametrize("offset", [0.0, 0.03, -0.07, 0.2])
def test_proposal_ends_on_the_bisection_grid_cell(fake_runs, offset):
    """The proposal's probes lie on bisection's grid of Ca values, so with a
    monotone verdict both searches end on the same grid cell."""
    sb, _ = study.search_bisect(TRIPLES, tol=0.02)
    sm, _ = study.search_mlp(TRIPLES, FakeNetwork(offset), tol=0.02, delta=0.06)
    h = study.grid_step(study.CA_MIN, study.CA_MAX, 0.02)
    assert h == pytest.approx(1.6 / 128)
    for b, m in zip(sb, sm):
        assert m.lo == pytest.approx(b.lo) and m.hi == pytest.approx(b.hi)
        for ca, _ in m.history:
            k = (ca - study.CA_MIN) / h
            assert abs(k - round(k)) < 1e-9


def test_bisection_at_another_wall_speed_and_range(monkeypatch):
    """The trend's second wall speed reaches every case of the search, and
    the search range follows its upper end."""
    seen = []

    def run_batch(cases, device=None, stats=None):
        seen.extend(c.uw for c in cases)
        return [study.Verdict(c.Ca > 2.45, 0.1, 30.0, 0, float("nan")) for c in cases]

    monkeypatch.setattr(study, "run_batch", run_batch)
    searches, _ = study.search_bisect([(0.0, 1.0, 0.7, 1)], tol=0.02, hi=2.7, uw=0.098)
    s = searches[0]
    assert seen and all(u == 0.098 for u in seen)
    assert s.lo <= 2.45 < s.hi and s.width <= 0.02
    p = study.case_params(study._case(s.triple, 2.0, 0, uw=0.098))
    p0 = study.case_params(study._case(s.triple, 2.0, 0))
    # the same Ca at a higher wall speed: the same viscosity times shear
    # rate, so a proportionally smaller matrix viscosity
    assert p.Uw == 0.098 and abs(p.eta_M * 0.098 - p0.eta_M * study.UW) < 1e-12


def test_blown_up_runs_count_as_breaking_and_are_listed(monkeypatch):
    """A run that blows up gives no verdict: the search treats it as
    breaking and lists its Ca, so a report can show which brackets rest on
    one."""
    def run_batch(cases, device=None, stats=None):
        return [study.Verdict(c.Ca > 1.5, 0.1, 30.0, 0, float("nan"), ok=c.Ca < 2.0) for c in cases]

    monkeypatch.setattr(study, "run_batch", run_batch)
    searches, stats = study.search_bisect([(2.0, 1.0, 0.7, 2)], tol=0.02)
    s = searches[0]
    assert s.diverged == [study.CA_MAX] and stats["diverged"] == 1
    assert (study.CA_MAX, True) in s.history
    assert s.lo <= 1.5 < s.hi and s.width <= 0.02


def test_cases_at_a_larger_gap():
    """At another gap W the box scales with it (x and y extents rounded to
    multiples of 8 and 4), R = (2R/W) W / 2, and a given Ca needs the same
    matrix viscosity (Ca = eta_M (2 U_w / W) R / sigma, so W cancels at a
    fixed 2R/W): the relaxation times, and with them the reachable Ca range,
    do not change with W."""
    c40 = study.Case(Ca=1.7, De=2.0, lam=1.0, conf=0.7, phase=2)
    c64 = study.Case(Ca=1.7, De=2.0, lam=1.0, conf=0.7, phase=2, w=64)
    p40, p64 = study.case_params(c40), study.case_params(c64)
    assert (p40.Lx, p40.Ly, p40.Lz) == (study.LX, study.LY, study.W)
    assert (p64.Lx, p64.Ly, p64.Lz) == (512, 72, 64)
    assert p64.R == 0.5 * 0.7 * 64
    assert abs(p64.eta_M - p40.eta_M) < 1e-12 and abs(p64.eta_P - p40.eta_P) < 1e-12
    # the emulsion time (in steps) grows with W at a fixed wall speed
    assert abs(study.tau_em(c64) / study.tau_em(c40) - 64 / 40) < 1e-12
