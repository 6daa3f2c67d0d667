"""Train the proposal network on solver runs and compare Ca_cr searches.

python -m paper_1411_2181_gb300.study_run --train 1024 --triples 16 --out report.json

1. ``--train`` cases drawn over (Ca, De, lambda, 2R/W, phase) are simulated
   in batches; their verdicts and shapes are the training set.
2. The network is trained by the CUDA kernels (AdamW, BF16 weights).
3. For ``--triples`` held-out (De, lambda, 2R/W, phase) triples (seed 5), Ca_cr
   is searched by plain bisection and with the network's bracket; both give
   brackets of width <= 0.02 confirmed by full runs.  The report lists, per
   mode, the number of full simulations, batched rounds and wall time, and
   per triple both brackets.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import mlp, study


def held_out_triples(n: int, seed: int = 5):
    rng = np.random.default_rng(seed)
    return [(float(rng.choice([0.0, 0.5, 1.0, 2.0])), float(rng.choice(study.LAMBDAS)),
             float(rng.uniform(study.CONF_MIN + 0.02, study.CONF_MAX - 0.02)), int(rng.choice([1, 2])))
            for _ in range(n)]


def CA_IN(s) -> bool:
    """Ca_cr strictly inside the search range (not at either end)."""
    return study.CA_MIN < 0.5 * (s.lo + s.hi) < study.CA_MAX


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=1024)
    ap.add_argument("--triples", type=int, default=16)
    ap.add_argument("--epochs", type=int, default=1500)
    ap.add_argument("--delta", type=float, default=0.06)
    ap.add_argument("--out", default=None)
    ap.add_argument("--params-out", default=None)
    ap.add_argument("--params-in", default=None, help="reuse a trained network (skips the training runs)")
    ap.add_argument("--trend", action="store_true",
                    help="only Ca_cr by bisection against the confinement 2R/W for Newtonian, DV and MV "
                         "droplets at De = 2, lambda = 1 (the trends of Figs. 2 and 4, reduced domains)")
    ap.add_argument("--trend-lambda", type=float, default=1.0, help="viscosity ratio of the --trend cases")
    a = ap.parse_args(argv)
    if a.trend:
        return trend(a.out, a.trend_lambda)

    report = {}
    t0 = time.perf_counter()
    net = mlp.MLP(max_batch=max(4096, a.train), bf16=True)
    if a.params_in:
        net.set_params(np.load(a.params_in))
        report["network"] = {"loaded": a.params_in}
    else:
        st_train = {}
        cases, verdicts = study.training_set(a.train, seed=100, stats=st_train)
        report["training_runs"] = dict(st_train, valid=len(cases), broken=int(sum(v.broken for v in verdicts)))
        X = study.features(cases)
        T, M = study.targets(verdicts)
        # hold out 1/8 of the runs to estimate the network's accuracy
        n_val = max(1, len(X) // 8)
        net.set_params(mlp.init_params(0))
        t1 = time.perf_counter()
        hist = net.fit(X[n_val:], T[n_val:], M[n_val:], epochs=a.epochs, lr=3e-3, batch=256)
        train_s = time.perf_counter() - t1
        yv = net.forward(X[:n_val])
        acc = float(np.mean((yv[:, 2] > 0) == (T[:n_val, 2] > 0.5)))
        d_err = float(np.sqrt(np.sum(M[:n_val] * (yv[:, 0] - T[:n_val, 0]) ** 2) / max(1.0, M[:n_val].sum())))
        report["network"] = {"epochs": a.epochs, "final_loss": hist[-1], "first_loss": hist[0],
                             "train_seconds": train_s, "val_breakup_accuracy": acc, "val_D_rmse": d_err}
    if a.params_out:
        np.save(a.params_out, net.get_params())

    triples = held_out_triples(a.triples)
    sb, stb = study.search_bisect(triples)
    sm, stm = study.search_mlp(triples, net, delta=a.delta)
    per = []
    agree = overlap = 0
    for b, m in zip(sb, sm):
        cb, cm = 0.5 * (b.lo + b.hi), 0.5 * (m.lo + m.hi)
        agree += abs(cb - cm) <= 0.01 + 1e-9
        overlap += max(b.lo, m.lo) <= min(b.hi, m.hi) + 1e-12
        per.append({"triple": b.triple, "bisect": [b.lo, b.hi, b.runs], "mlp": [m.lo, m.hi, m.runs]})
    keys = ("runs", "rounds", "seconds", "lattice_updates", "diverged")
    report["bisect"] = {k: stb.get(k, 0) for k in keys}
    report["mlp"] = {k: stm.get(k, 0) for k in keys}
    report["in_range"] = int(sum(CA_IN(b) for b in sb))
    report["agree_within_0.01"] = f"{agree}/{len(triples)}"
    report["brackets_consistent"] = f"{overlap}/{len(triples)}"
    report["per_triple"] = per
    report["total_seconds"] = time.perf_counter() - t0
    txt = json.dumps(report, indent=1)
    print(txt)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(txt)
    return report


def trend(out=None, lam=1.0):
    """Ca_cr (bisection, bracket width 0.02) for Newtonian (De = 0), droplet-
    and matrix-viscoelastic (De = 2) droplets at viscosity ratio lam and 2R/W in
    {0.6, 0.7, 0.8} on the study's reduced domains.  Sec. 3 reports, at the
    paper's sizes, that confinement raises Ca_cr, droplet viscoelasticity
    raises it further and matrix viscoelasticity lowers it."""
    kinds = (("newtonian", 0.0, 1), ("DV", 2.0, 1), ("MV", 2.0, 2))
    confs = (0.6, 0.7, 0.8)
    triples = [(De, lam, conf, phase) for conf in confs for _, De, phase in kinds]
    t0 = time.perf_counter()
    sb, st = study.search_bisect(triples)
    rows = {}
    for (name, _, _), i in zip(kinds * len(confs), range(len(triples))):
        s = sb[i]
        rows.setdefault(name, []).append({"2R/W": s.triple[2], "Ca_cr": 0.5 * (s.lo + s.hi),
                                          "bracket": [s.lo, s.hi], "runs": s.runs})
    report = {"lambda": lam, "trend": rows, "runs": st.get("runs", 0), "rounds": st.get("rounds", 0),
              "diverged": st.get("diverged", 0), "seconds": time.perf_counter() - t0}
    txt = json.dumps(report, indent=1)
    print(txt)
    if out:
        with open(out, "w") as fh:
            fh.write(txt)
    return report


if __name__ == "__main__":
    main()
