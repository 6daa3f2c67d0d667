"""Collect solver runs, train the proposal network, compare Ca_cr searches.

The three steps can run in separate processes (the collection is the
expensive one: a full simulation per case):

  python -m paper_1411_2181_gb300.study_run collect --n 512 --seed 100 --out runs_100.jsonl
  python -m paper_1411_2181_gb300.study_run train --data runs_100.jsonl,runs_101.jsonl --params-out net.npy
  python -m paper_1411_2181_gb300.study_run search --params net.npy --triples 16 --out report.json
  python -m paper_1411_2181_gb300.study_run trend --out trend.json

collect  simulates cases drawn by study.sample_cases (batched full runs) and
         appends one JSON line per run: the case and its verdict (break-up,
         steady D and theta, necks, break-up time, blown up or not);
train    fits the network to the collected runs with the CUDA kernels
         (AdamW, BF16 weights, FP32 accumulation), holding out one run in
         eight to report its accuracy, and saves the FP32 parameters;
search   searches Ca_cr for held-out (De, lambda, 2R/W) triples of the
         matrix-viscoelastic family (seed 5), by plain bisection and with the
         network's bracket; both end with brackets of width <= 0.02 whose
         ends are full-run verdicts.  The report lists, per mode, the full
         simulations, batched rounds and wall time, and per triple both
         brackets;
trend    Ca_cr by bisection against the confinement for Newtonian, droplet-
         and matrix-viscoelastic droplets (the trends of Figs. 2 and 4);
breakup  how given cases break: necks before break-up, break-up time and
         the number of fragments (binary or multiple break-up, Sec. 3).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import study

HELD_OUT_DE = (1.0, 1.5, 2.0)


def held_out_triples(n: int, seed: int = 5):
    """(De, lambda, 2R/W, phase) of the matrix-viscoelastic family, whose
    Ca_cr lies inside the search range at the study's resolution; the
    confinements are continuous draws, so no triple equals a training
    case's."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        t = (float(rng.choice(HELD_OUT_DE)), float(rng.choice(study.LAMBDAS)),
             float(round(rng.uniform(study.CONF_MIN + 0.02, study.CONF_MAX - 0.02), 4)), 2)
        if t not in out:
            out.append(t)
    return out


def interior(s) -> bool:
    """Ca_cr strictly inside the search range (not at either end)."""
    return study.CA_MIN < 0.5 * (s.lo + s.hi) < study.CA_MAX


def _case_json(c, v):
    return {"Ca": c.Ca, "De": c.De, "lam": c.lam, "conf": c.conf, "L2": c.L2, "phase": c.phase, "seed": c.seed,
            "broken": bool(v.broken), "D": float(v.D), "theta": float(v.theta), "necks": int(v.necks),
            "t_break": None if v.t_break != v.t_break else float(v.t_break), "ok": bool(v.ok)}


def collect(n: int, seed: int, out: str, batch: int = 64, mv_ca_from: float | None = None):
    """Simulate n training cases; one JSON line per run (written per batch)."""
    stats = {}
    t0 = time.perf_counter()
    written = [0]

    def progress(cases, verdicts):
        with open(out, "a") as fh:
            for c, v in zip(cases[written[0]:], verdicts[written[0]:]):
                fh.write(json.dumps(_case_json(c, v)) + "\n")
        written[0] = len(verdicts)

    open(out, "w").close()
    study.training_set(n, seed=seed, batch=batch, stats=stats, progress=progress, mv_ca_from=mv_ca_from)
    stats["wall_seconds"] = time.perf_counter() - t0
    print(json.dumps({"collected": written[0], "seed": seed, "stats": stats}))
    return stats


def load_runs(paths):
    cases, verdicts = [], []
    for p in paths:
        with open(p) as fh:
            for line in fh:
                d = json.loads(line)
                if not d["ok"]:
                    continue
                cases.append(study.Case(Ca=d["Ca"], De=d["De"], lam=d["lam"], conf=d["conf"], L2=d["L2"],
                                        phase=d["phase"], seed=d["seed"]))
                tb = d["t_break"]
                verdicts.append(study.Verdict(d["broken"], d["D"], d["theta"], d["necks"],
                                              float("nan") if tb is None else tb))
    return cases, verdicts


def train(paths, epochs: int = 1500, params_out: str | None = None, seed: int = 0):
    from . import mlp
    cases, verdicts = load_runs(paths)
    X = study.features(cases)
    T, M = study.targets(verdicts)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(X))
    X, T, M = X[perm], T[perm], M[perm]
    n_val = max(1, len(X) // 8)
    net = mlp.MLP(max_batch=max(4096, len(X)), bf16=True)
    net.set_params(mlp.init_params(seed))
    t1 = time.perf_counter()
    hist = net.fit(X[n_val:], T[n_val:], M[n_val:], epochs=epochs, lr=3e-3, batch=256)
    train_s = time.perf_counter() - t1
    yv = net.forward(X[:n_val])
    acc = float(np.mean((yv[:, 2] > 0) == (T[:n_val, 2] > 0.5)))
    d_err = float(np.sqrt(np.sum(M[:n_val] * (yv[:, 0] - T[:n_val, 0]) ** 2) / max(1.0, M[:n_val].sum())))
    info = {"runs": int(len(X)), "broken": int(T[:, 2].sum()), "epochs": epochs, "first_loss": hist[0],
            "final_loss": hist[-1], "train_seconds": train_s, "val_runs": n_val,
            "val_breakup_accuracy": acc, "val_D_rmse": d_err}
    if params_out:
        np.save(params_out, net.get_params())
    print(json.dumps(info))
    return net, info


def compare(net, triples, delta: float = 0.06):
    """Both searches over the same triples; the comparison of the report."""
    sb, stb = study.search_bisect(triples)
    sm, stm = study.search_mlp(triples, net, delta=delta)
    per = []
    agree = overlap = 0
    for b, m in zip(sb, sm):
        cb, cm = 0.5 * (b.lo + b.hi), 0.5 * (m.lo + m.hi)
        agree += abs(cb - cm) <= 0.01 + 1e-9
        overlap += max(b.lo, m.lo) <= min(b.hi, m.hi) + 1e-12
        per.append({"triple": b.triple, "bisect": [b.lo, b.hi, b.runs], "mlp": [m.lo, m.hi, m.runs],
                    "interior": bool(interior(b))})
    keys = ("runs", "rounds", "seconds", "lattice_updates", "diverged")
    return {"bisect": {k: stb.get(k, 0) for k in keys}, "mlp": {k: stm.get(k, 0) for k in keys},
            "interior": int(sum(interior(b) for b in sb)), "triples": len(triples),
            "agree_within_0.01": int(agree), "brackets_consistent": int(overlap), "delta": delta,
            "per_triple": per}


def search(params: str, n_triples: int, out: str | None, delta: float = 0.06, train_info: dict | None = None):
    from . import mlp
    net = mlp.MLP(max_batch=4096, bf16=True)
    net.set_params(np.load(params))
    t0 = time.perf_counter()
    rep = compare(net, held_out_triples(n_triples), delta=delta)
    rep["total_seconds"] = time.perf_counter() - t0
    rep["regime"] = {"W": study.W, "Lx": study.LX, "Ly": study.LY, "Uw": study.UW, "G": study.G_STUDY,
                     "Ca_range": [study.CA_MIN, study.CA_MAX], "t_max_tem": study.T_MAX_TEM,
                     "conf_range": [study.CONF_MIN, study.CONF_MAX]}
    if train_info:
        rep["network"] = train_info
    _emit(rep, out)
    return rep


def trend(out=None, lam=1.0, confs=(0.6, 0.7, 0.8), uw=study.UW, ca_max=study.CA_MAX, de=2.0, w=study.W,
          kinds=("newtonian", "DV", "MV")):
    """Ca_cr (bisection, bracket width 0.02) for Newtonian (De = 0), droplet-
    and matrix-viscoelastic (De = de) droplets at viscosity ratio lam against
    2R/W on the study's domains.  Sec. 3 reports, at the paper's sizes, that
    droplet viscoelasticity raises Ca_cr and matrix viscoelasticity lowers
    it, more so under strong confinement.  A higher wall speed uw reaches a
    higher Ca at the same relaxation times (Ca is proportional to the shear
    rate), as in the paper's protocol of raising the wall speed.  A larger
    gap w (the box scaled with it) resolves the droplet and its interface
    more finely at the same range of Ca."""
    kinds = tuple(k for k in (("newtonian", 0.0, 1), ("DV", de, 1), ("MV", de, 2)) if k[0] in kinds)
    triples = [(De, lam, conf, phase) for conf in confs for _, De, phase in kinds]
    t0 = time.perf_counter()
    sb, st = study.search_bisect(triples, hi=ca_max, uw=uw, w=w)
    rows = {}
    for i, s in enumerate(sb):
        name = kinds[i % len(kinds)][0]
        lo_open = s.lo == s.hi == ca_max
        rows.setdefault(name, []).append({"2R/W": s.triple[2], "bracket": [s.lo, s.hi],
                                          "Ca_cr": (None if lo_open else 0.5 * (s.lo + s.hi)),
                                          "stable_over_range": bool(lo_open), "runs": s.runs,
                                          "diverged_at": sorted(s.diverged)})
    rep = {"lambda": lam, "trend": rows, "runs": st.get("runs", 0), "rounds": st.get("rounds", 0),
           "diverged": st.get("diverged", 0), "seconds": time.perf_counter() - t0,
           "Ca_range": [study.CA_MIN, ca_max], "Uw": uw, "De": de, "W": w,
           "box": [getattr(study.case_params(study._case(triples[0], 1.0, 0, uw=uw, w=w)), k)
                   for k in ("Lx", "Ly", "Lz")]}
    _emit(rep, out)
    return rep


def breakup(specs, out=None, uw=study.UW, w=study.W, every_tem=0.25):
    """Break-up details (study.breakup_details) of cases given as
    (De, lambda, 2R/W, phase, Ca), run as one batch."""
    cases = [study.Case(Ca=ca, De=de, lam=lam, conf=conf, phase=int(ph), seed=7, uw=uw, w=w)
             for de, lam, conf, ph, ca in specs]
    t0 = time.perf_counter()
    rep = {"W": w, "Uw": uw, "every_tem": every_tem, "cases": study.breakup_details(cases, every_tem=every_tem),
           "seconds": time.perf_counter() - t0}
    _emit(rep, out)
    return rep


def _emit(rep, out):
    txt = json.dumps(rep, indent=1)
    print(txt)
    if out:
        with open(out, "w") as fh:
            fh.write(txt)


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--n", type=int, default=512)
    c.add_argument("--seed", type=int, default=100)
    c.add_argument("--out", required=True)
    c.add_argument("--mv-ca-from", type=float, default=None,
                   help="lower end of the matrix-viscoelastic cases' Ca (default: the search range's)")
    t = sub.add_parser("train")
    t.add_argument("--data", required=True, help="comma-separated collect outputs")
    t.add_argument("--epochs", type=int, default=1500)
    t.add_argument("--params-out", required=True)
    s = sub.add_parser("search")
    s.add_argument("--params", required=True)
    s.add_argument("--triples", type=int, default=16)
    s.add_argument("--delta", type=float, default=0.06)
    s.add_argument("--out", default=None)
    s.add_argument("--train-info", default=None, help="JSON file of the train step, copied into the report")
    r = sub.add_parser("trend")
    r.add_argument("--out", default=None)
    r.add_argument("--lam", type=float, default=1.0)
    r.add_argument("--uw", type=float, default=study.UW, help="wall speed (lattice units)")
    r.add_argument("--ca-max", type=float, default=study.CA_MAX)
    r.add_argument("--de", type=float, default=2.0, help="Deborah number of the DV and MV droplets")
    r.add_argument("--w", type=int, default=study.W, help="gap W (the box scales with it)")
    r.add_argument("--kinds", default="newtonian,DV,MV")
    b = sub.add_parser("breakup")
    b.add_argument("--case", action="append", required=True, help="De,lambda,2R/W,phase,Ca (repeatable)")
    b.add_argument("--uw", type=float, default=study.UW)
    b.add_argument("--w", type=int, default=study.W)
    b.add_argument("--every", type=float, default=0.25, help="observation interval in emulsion times")
    b.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    if a.cmd == "collect":
        return collect(a.n, a.seed, a.out, mv_ca_from=a.mv_ca_from)
    if a.cmd == "train":
        return train(a.data.split(","), a.epochs, a.params_out)
    if a.cmd == "search":
        info = json.load(open(a.train_info)) if a.train_info else None
        return search(a.params, a.triples, a.out, a.delta, info)
    if a.cmd == "breakup":
        return breakup([tuple(float(x) for x in c.split(",")) for c in a.case], a.out, uw=a.uw, w=a.w,
                       every_tem=a.every)
    return trend(a.out, a.lam, uw=a.uw, ca_max=a.ca_max, de=a.de, w=a.w, kinds=tuple(a.kinds.split(",")))


if __name__ == "__main__":
    main()
