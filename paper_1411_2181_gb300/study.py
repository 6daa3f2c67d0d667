"""Critical Capillary number search (Sec. 3) with and without the learned
proposal.

Sec. 3 defines Ca_cr through the largest wall velocity at which the droplet
stays stable and the smallest at which it breaks.  Here a case is the
tuple (Ca, De, lambda, 2R/W, L^2, viscoelastic phase); Ca varies through the
matrix viscosity at a fixed wall speed (the paper varies the wall speed at a
fixed viscosity: the same Ca at a different Reynolds number; the wall speed
here is capped by the lattice Mach limit).  A verdict is one full
simulation of the case on the GPU:
  broken  - the break-up flag (two separated occupied x-runs, each >= 1% of
            the volume) was set at an observation before t_max;
  stable  - otherwise.
Cases are simulated in batches (one persistent launch per step advances
every case of the batch).

Two search modes over held-out (De, lambda, 2R/W, phase) triples:
  bisect  - bracket [Ca_lo, Ca_hi] = [CA_MIN, CA_MAX] checked by two runs, then
            halved until Ca_hi - Ca_lo <= tol;
  mlp     - the network's break-up logit over a Ca grid gives Ca* and the
            bracket Ca* -/+ delta; both ends are verified by full runs (and
            the bracket is moved outwards until they are stable / broken),
            then halved until the width is <= tol.  A case predicted stable
            (breaking) over the whole range is first run at that end only.
Every verdict in both modes comes from a full simulation; the network only
chooses which simulations to run.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import configs, synth
from .params import Params

# Study regime (lattice units).  Small droplets dissolve into the matrix
# through the Shan-Chen miscibility, faster at high viscosity (the mutual
# diffusivity grows with tau - 1/2); the study therefore uses a stronger
# coupling G = 3.8 (flat-interface coexistence densities 1.05503 / 0.01288,
# sigma = 0.0985 from the oracle's Laplace fit; both recorded in
# tests/golden/shan_chen_constants.txt), droplets with 2R/W in
# [0.6, 0.8] at W = 40, and varies Ca through the matrix viscosity at the
# wall speed 0.08, which keeps every BGK relaxation time below about 13
# (runs with tau above about 13 in the droplet diverge at this coupling).
# The box is 320 cells long (20-27 R): a droplet near break-up stretches to
# 12-16 R, and in a shorter periodic box it joins its own image and can
# never separate into fragments.  At this resolution matrix-viscoelastic
# droplets break inside [CA_MIN, CA_MAX]; Newtonian and droplet-
# viscoelastic ones (thick diffuse interfaces resist necking, and a higher
# Ca would need a relaxation time beyond the stable range) stay intact up
# to Ca = 2.
G_STUDY = 3.8
RHO_IN_STUDY, RHO_OUT_STUDY = 1.05503, 0.01288
SIGMA_STUDY = 0.09854
W = 40
LX, LY = 320, 44
CA_MIN, CA_MAX = 0.6, 2.2
CA_MID, CA_HALF = 1.4, 0.8         # network input scaling of Ca
UW = 0.08
CONF_MIN, CONF_MAX = 0.6, 0.8
LAMBDAS = (0.5, 1.0)
T_MAX_TEM = 30.0      # simulated time in emulsion times
OBS_EVERY_TEM = 0.5


@dataclass
class Case:
    Ca: float
    De: float
    lam: float
    conf: float        # 2R/W
    L2: float = 100.0
    phase: int = 1     # 1 droplet viscoelastic, 2 matrix viscoelastic
    seed: int = 0
    uw: float = UW     # wall speed (the trend at a second wall speed; the network's cases keep UW)
    w: int = W         # gap; the box scales with it (the trend at a finer resolution)


@dataclass
class Verdict:
    broken: bool
    D: float
    theta: float
    necks: int
    t_break: float     # in emulsion times, nan if stable
    ok: bool = True


def case_params(c: Case) -> Params:
    """Lattice parameters of a case: its wall speed, eta_M from Ca (Sec. 1),
    tau_P from De (Eq. 8), emulsion time R eta_M / sigma (Eq. 9)."""
    R = 0.5 * c.conf * c.w
    lx, ly = (LX, LY) if c.w == W else (int(round(LX * c.w / W / 8)) * 8, int(round(LY * c.w / W / 4)) * 4)
    return configs.make_params(lx, ly, c.w, R, Ca=c.Ca, De=c.De, lam=c.lam, beta=0.4, L2=c.L2, phase=c.phase,
                               Uw=c.uw, G=G_STUDY, sigma=SIGMA_STUDY, rho_in=RHO_IN_STUDY,
                               rho_out=RHO_OUT_STUDY)


def tau_em(c: Case) -> float:
    p = case_params(c)
    return p.R * p.eta_M / p.sigma


def features(cases) -> np.ndarray:
    """Scaled network inputs: (Ca, De, ln lambda, 2R/W, ln L^2, phase)."""
    X = np.array([[(c.Ca - CA_MID) / CA_HALF, (c.De - 1.0), math.log(c.lam) / math.log(2.0), (c.conf - 0.7) / 0.1,
                   (math.log(c.L2) - math.log(200.0)) / math.log(4.0), -1.0 if c.phase == 1 else 1.0]
                  for c in cases], dtype=np.float32)
    return X


def targets(verdicts) -> tuple[np.ndarray, np.ndarray]:
    T = np.array([[v.D, v.theta / 90.0, 1.0 if v.broken else 0.0, v.necks / 4.0] for v in verdicts], np.float32)
    M = np.array([0.0 if v.broken else 1.0 for v in verdicts], np.float32)
    return T, M


def run_batch(cases: list[Case], device=None, stats: dict | None = None) -> list[Verdict]:
    """Simulate every case to t_max (or until all broke); one verdict each."""
    import torch
    from . import lbfe
    ps = [case_params(c) for c in cases]
    tem = [p.R * p.eta_M / p.sigma for p in ps]
    stream = torch.cuda.Stream(device)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        s = lbfe.Solver(ps, device=device, stream=stream)
        # one launch shape for every batch: the 8-row one-cell kernel (the
        # fastest FP32 shape), z-chunks fitted to the batch.  The z-chunk
        # does not change a cell's arithmetic, the kernel variant and tile
        # height can (FP32 rounding), and a verdict near the threshold must
        # not depend on which batch the case ran in
        s.tune(8, 0, 0)
        for k, (c, p) in enumerate(zip(cases, ps)):
            s.init(k, synth.droplet_densities(p.Lx, p.Ly, p.Lz, p.R, p.rho_in, p.rho_out, 1e-4, seed=c.seed))
        n = len(cases)
        broken = [False] * n
        ok = [True] * n
        last = [None] * n
        necks = [0] * n
        t_break = [float("nan")] * n
        # each case is observed on its own schedule -- every OBS_EVERY_TEM of
        # its emulsion time, up to T_MAX_TEM -- so that its verdict does not
        # depend on the other cases of the batch; the batch advances from
        # one observation to the next
        every = [max(1, int(round(OBS_EVERY_TEM * t))) for t in tem]
        last_obs = [int(math.ceil(T_MAX_TEM * t / e)) * e for t, e in zip(tem, every)]
        nxt = list(every)
        steps = 0
        while True:
            live = [k for k in range(n) if ok[k] and not broken[k] and nxt[k] <= last_obs[k]]
            if not live:
                break
            target = min(nxt[k] for k in live)
            s.step(target - steps)
            steps = target
            for k in live:
                if nxt[k] != steps:
                    continue
                nxt[k] += every[k]
                ob = s.observables(k, raise_on_diverged=False)
                if ob["flags"]:
                    ok[k] = False          # this instance blew up: no verdict
                    continue
                if ob["broken"]:
                    broken[k] = True
                    t_break[k] = steps / tem[k]
                else:
                    last[k] = ob
                    necks[k] = max(necks[k], ob["necks"])
        torch.cuda.synchronize()
        s.close()
    if stats is not None:
        stats["runs"] = stats.get("runs", 0) + len(cases)
        stats["batches"] = stats.get("batches", 0) + 1
        stats["seconds"] = stats.get("seconds", 0.0) + time.perf_counter() - t0
        stats["lattice_updates"] = stats.get("lattice_updates", 0) + steps * sum(p.N for p in ps)
    out = []
    for k in range(len(cases)):
        ob = last[k] or {"D": 0.0, "theta_deg": 0.0}
        out.append(Verdict(broken[k], ob["D"], ob["theta_deg"], necks[k], t_break[k], ok[k]))
    return out


def breakup_details(cases: list[Case], device=None, every_tem: float = 0.25, after_tem: float = 3.0) -> list[dict]:
    """How each case breaks (Sec. 3: binary break-up, or multiple necks and
    equal daughter droplets under strong confinement): observed every
    every_tem emulsion times up to T_MAX_TEM, and for after_tem more once it
    broke.  Per case: the largest neck count before break-up, the break-up
    time, the fragment count at break-up and the largest one after it, and
    the fragment count at every observation from the break-up on."""
    import torch
    from . import lbfe
    ps = [case_params(c) for c in cases]
    tem = [p.R * p.eta_M / p.sigma for p in ps]
    every = [max(1, int(round(every_tem * t))) for t in tem]
    out = [{"case": c.__dict__.copy(), "necks_before": 0, "t_break": None, "fragments_at_break": 0,
            "fragments_max": 0, "fragments_after": [], "ok": True} for c in cases]
    end = [int(math.ceil(T_MAX_TEM * t / e)) * e for t, e in zip(tem, every)]
    stream = torch.cuda.Stream(device)
    with torch.cuda.stream(stream):
        s = lbfe.Solver(ps, device=device, stream=stream)
        s.tune(8, 0, 0)
        for k, (c, p) in enumerate(zip(cases, ps)):
            s.init(k, synth.droplet_densities(p.Lx, p.Ly, p.Lz, p.R, p.rho_in, p.rho_out, 1e-4, seed=c.seed))
        nxt, steps = list(every), 0
        while True:
            live = [k for k in range(len(cases)) if out[k]["ok"] and nxt[k] <= end[k]]
            if not live:
                break
            target = min(nxt[k] for k in live)
            s.step(target - steps)
            steps = target
            for k in live:
                if nxt[k] != steps:
                    continue
                nxt[k] += every[k]
                ob = s.observables(k, raise_on_diverged=False)
                o = out[k]
                if ob["flags"]:
                    o["ok"] = False
                    continue
                if o["t_break"] is None:
                    if ob["broken"]:
                        o["t_break"] = steps / tem[k]
                        o["fragments_at_break"] = o["fragments_max"] = ob["fragments"]
                        o["fragments_after"].append(ob["fragments"])
                        end[k] = min(end[k], steps + int(math.ceil(after_tem * tem[k] / every[k])) * every[k])
                    else:
                        o["necks_before"] = max(o["necks_before"], ob["necks"])
                else:
                    o["fragments_max"] = max(o["fragments_max"], ob["fragments"])
                    o["fragments_after"].append(ob["fragments"])
        torch.cuda.synchronize()
        s.close()
    return out


DE_TRAIN = (0.0, 0.5, 1.0, 1.5, 2.0)


def sample_cases(n: int, seed: int, mv_ca_from: float | None = None) -> list[Case]:
    """Training cases.  Seven in ten are matrix-viscoelastic, with Ca
    uniform from mv_ca_from (default CA_MIN) to CA_MAX: their break-up
    happens inside the range at this resolution, where the network's logit
    must cross; the rest cover Newtonian and droplet-viscoelastic droplets
    over the whole range (stable there)."""
    rng = np.random.default_rng(seed)
    lo_mv = CA_MIN if mv_ca_from is None else mv_ca_from
    cs = []
    for k in range(n):
        mv = rng.uniform() < 0.7
        if mv:
            ca = rng.uniform(lo_mv, CA_MAX)
            De, phase = float(rng.choice(DE_TRAIN[1:])), 2
        else:
            ca = rng.uniform(CA_MIN, CA_MAX)
            De, phase = float(rng.choice(DE_TRAIN)), 1
        cs.append(Case(Ca=float(ca), De=De, lam=float(rng.choice(LAMBDAS)),
                       conf=float(rng.uniform(CONF_MIN, CONF_MAX)), L2=100.0, phase=phase,
                       seed=int(rng.integers(0, 2 ** 31))))
    return cs


def training_set(n: int, seed: int = 100, batch: int = 64, device=None, stats=None, progress=None,
                 mv_ca_from: float | None = None):
    """Simulate n sampled cases; batches hold cases of similar Ca (similar
    emulsion times, so that few steps go to cases already finished).
    Returns the cases and verdicts of the runs that did not blow up."""
    cases = sorted(sample_cases(n, seed, mv_ca_from), key=lambda c: c.Ca)
    verdicts = []
    for s in range(0, n, batch):
        verdicts += run_batch(cases[s:s + batch], device=device, stats=stats)
        if progress:
            progress(cases[:len(verdicts)], verdicts)
    keep = [k for k, v in enumerate(verdicts) if v.ok]
    cases = [cases[k] for k in keep]
    verdicts = [verdicts[k] for k in keep]
    return cases, verdicts


@dataclass
class Search:
    triple: tuple
    lo: float
    hi: float
    runs: int = 0
    history: list = field(default_factory=list)
    diverged: list = field(default_factory=list)   # Ca values whose run blew up (counted as breaking)

    @property
    def width(self):
        return self.hi - self.lo


def _case(triple, Ca, seed, **case_kw):
    De, lam, conf, phase = triple
    return Case(Ca=Ca, De=De, lam=lam, conf=conf, phase=phase, seed=seed, **case_kw)


def _verdict_round(searches, cas, device, stats, seed, case_kw=None):
    """One batched round: a full run for every (search, Ca) pair."""
    pairs = [(s, ca) for s, lst in zip(searches, cas) for ca in lst]
    if not pairs:
        return {}
    vs = run_batch([_case(s.triple, ca, seed, **(case_kw or {})) for s, ca in pairs], device=device, stats=stats)
    res = {}
    for (s, ca), v in zip(pairs, vs):
        s.runs += 1
        # a run that blew up gives no verdict; it is counted as breaking (the
        # search then stays below the unstable range) and reported
        br = v.broken or not v.ok
        if not v.ok:
            stats["diverged"] = stats.get("diverged", 0) + 1
            s.diverged.append(ca)
        s.history.append((ca, br))
        res[(id(s), ca)] = br
    return res


def grid_step(lo: float, hi: float, tol: float) -> float:
    """Spacing of the Ca values plain bisection of [lo, hi] can visit before
    its bracket is <= tol wide: (hi - lo) / 2^k with the smallest such k."""
    return (hi - lo) / 2 ** math.ceil(math.log2((hi - lo) / tol) - 1e-12)


def _on_grid(x: float, lo: float, h: float) -> float:
    return lo + round((x - lo) / h) * h


def _bisect_rounds(searches, tol, device, stats, seed, grid=None, case_kw=None):
    """Halve every open bracket until it is <= tol wide.  With a grid
    (lo, h) the probe is the grid point nearest the bracket's middle, so
    that brackets on the grid stay on it."""
    while True:
        act = [s for s in searches if s.width > tol + 1e-12]
        if not act:
            return
        if grid:
            g0, h = grid
            mids = []
            for s in act:
                k_lo, k_hi = round((s.lo - g0) / h), round((s.hi - g0) / h)
                mids.append([g0 + ((k_lo + k_hi) // 2) * h])
        else:
            mids = [[0.5 * (s.lo + s.hi)] for s in act]
        res = _verdict_round(act, mids, device, stats, seed, case_kw)
        for s, (m,) in zip(act, mids):
            if res[(id(s), m)]:
                s.hi = m
            else:
                s.lo = m
        stats["rounds"] = stats.get("rounds", 0) + 1


def search_bisect(triples, tol=0.02, lo=CA_MIN, hi=CA_MAX, device=None, seed=7, **case_kw):
    """Plain bisection: verify the initial bracket, then halve it (the
    midpoints are the grid points lo + k (hi - lo) / 2^n, computed as such).
    case_kw: Case fields other than the triple's (wall speed uw, gap w)."""
    stats = {}
    searches = [Search(t, lo, hi) for t in triples]
    res = _verdict_round(searches, [[lo, hi]] * len(searches), device, stats, seed, case_kw)
    stats["rounds"] = 1
    for s in searches:
        if res[(id(s), lo)]:
            s.hi = s.lo = lo          # breaks already at the lower end
        elif not res[(id(s), hi)]:
            s.lo = s.hi = hi          # stable at the upper end
    _bisect_rounds(searches, tol, device, stats, seed, grid=(lo, grid_step(lo, hi, tol)), case_kw=case_kw)
    return searches, stats


def search_mlp(triples, net, tol=0.02, delta=0.04, lo=CA_MIN, hi=CA_MAX, device=None, seed=7):
    """Network-proposed bracket Ca* -/+ delta: both ends are verified by full
    runs; an end that contradicts the bracket (the lower end breaks, or the
    upper end stays stable) becomes the other end and the bracket moves by
    2 delta in that direction, until both ends hold.  Then it is halved.
    Every probe lies on the grid of Ca values plain bisection of [lo, hi]
    visits (Ca* and delta rounded to it, delta to at least one step), so
    that where the verdicts are monotone in Ca both searches end on the
    same grid cell."""
    stats = {"rounds": 0}
    h = grid_step(lo, hi, tol)
    delta = max(h, round(delta / h) * h)
    grid = np.linspace(lo, hi, 341)
    searches, ok = [], {}
    for t in triples:
        X = features([_case(t, float(ca), 0) for ca in grid])
        logit = net.forward(X)[:, 2]
        above = np.nonzero(logit > 0)[0]
        if len(above) == 0:
            # predicted stable over the whole range: one run at the upper end
            s = Search(t, hi, hi)
            ok[id(s)] = [False, True]
        elif above[0] == 0:
            # predicted to break over the whole range: one run at the lower end
            s = Search(t, lo, lo)
            ok[id(s)] = [True, False]
        else:
            ca_star = _on_grid(float(grid[above[0]]), lo, h)
            s = Search(t, max(lo, _on_grid(ca_star - delta, lo, h)), min(hi, _on_grid(ca_star + delta, lo, h)))
            ok[id(s)] = [False, False]   # lower end stable / upper end broken verified
        searches.append(s)
    pending = list(searches)
    while pending:
        cas = [sorted({e for e, done in ((s.lo, ok[id(s)][0]), (s.hi, ok[id(s)][1])) if not done})
               for s in pending]
        res = _verdict_round(pending, cas, device, stats, seed)
        stats["rounds"] += 1
        nxt = []
        for s in pending:
            f = ok[id(s)]
            r_lo = None if f[0] else res[(id(s), s.lo)]
            r_hi = None if f[1] else res[(id(s), s.hi)]
            if s.lo == s.hi:                      # a single predicted end was run
                if r_lo is False:                 # stable at the upper limit: Ca_cr >= hi
                    f[0] = f[1] = True
                    continue
                if r_hi is True:                  # breaks at the lower limit: Ca_cr <= lo
                    f[0] = f[1] = True
                    continue
            if r_lo is True:                      # breaks at the lower end: Ca_cr is below it
                s.hi, f[1] = s.lo, True
                if s.lo <= lo:
                    s.lo, f[0] = lo, True
                else:
                    s.lo, f[0] = max(lo, _on_grid(s.lo - 2 * delta, lo, h)), False
            elif r_hi is False:                   # stable at the upper end: Ca_cr is above it
                s.lo, f[0] = s.hi, True
                if s.hi >= hi:
                    s.hi, f[1] = hi, True
                else:
                    s.hi, f[1] = min(hi, _on_grid(s.hi + 2 * delta, lo, h)), False
            else:
                if r_lo is False:
                    f[0] = True
                if r_hi is True:
                    f[1] = True
            if not (f[0] and f[1]):
                nxt.append(s)
        pending = nxt
    _bisect_rounds(searches, tol, device, stats, seed, grid=(lo, h))
    return searches, stats
