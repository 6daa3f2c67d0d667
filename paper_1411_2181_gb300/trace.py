"""Time series of a run's observables as JSON lines: one object per
observation with the step, t / tau_em, the deformation D and orientation
theta (Secs. 1 and 3), the projected length L_p / 2R (Sec. 3), the neck
count, the break-up flag and the mass of each component."""
from __future__ import annotations

import json

FIELDS = ("step", "t_over_tem", "D", "theta_deg", "Lp_over_2R", "necks", "broken", "mass")


def record(obs: dict, k: int = 0) -> dict:
    """The logged subset of one observables dictionary (``Solver.observables``)."""
    row = {"instance": k}
    for f in FIELDS:
        v = obs[f]
        row[f] = list(v) if isinstance(v, tuple) else v
    return row


def run_logged(solver, k: int, steps: int, every: int, path: str) -> list[dict]:
    """Advance instance k of ``solver`` by ``steps`` time steps, observing it
    before the first step and after every ``every`` steps (and at the end),
    and append one JSON line per observation to ``path``.  A diverged
    instance is logged (its flags are in the observables) and stops the run."""
    if every <= 0 or steps < 0:
        raise ValueError("every must be positive and steps non-negative")
    rows = []
    done = 0
    with open(path, "a") as fh:
        while True:
            o = solver.observables(k, raise_on_diverged=False)
            row = record(o, k)
            fh.write(json.dumps(row) + "\n")
            rows.append(row)
            if done >= steps or o.get("flags", 0):
                break
            n = min(every, steps - done)
            solver.step(n)
            done += n
    return rows


def main(argv=None):
    """Log the 192 x 96 x 80 matrix-viscoelastic droplet (W = 80, R = 16,
    De = 1, L^2 = 100) at each requested Ca, one JSON line per observation
    with the Ca added.  --coupling study runs it at the Ca_cr study's
    Shan-Chen coupling G = 3.8 (with its coexistence densities and sigma)
    instead of G = 3.1, at which an R = 16 droplet dissolves into the matrix
    within about 10^4 steps:

        python -m paper_1411_2181_gb300.trace --ca 0.1,0.2,0.3 --steps 20000 --every 200 --out ts.jsonl
    """
    import argparse

    from . import configs, lbfe
    ap = argparse.ArgumentParser()
    ap.add_argument("--ca", default="0.1,0.2,0.3")
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--every", type=int, default=200)
    ap.add_argument("--out", required=True)
    ap.add_argument("--coupling", choices=("default", "study"), default="default")
    a = ap.parse_args(argv)
    open(a.out, "w").close()
    for ca in (float(x) for x in a.ca.split(",")):
        if a.coupling == "study":
            from . import study, synth
            p = configs.make_params(192, 96, 80, 16.0, Ca=ca, De=1.0, lam=1.0, beta=0.4, L2=100.0, phase=2,
                                    Uw=0.02, G=study.G_STUDY, sigma=study.SIGMA_STUDY,
                                    rho_in=study.RHO_IN_STUDY, rho_out=study.RHO_OUT_STUDY)
            rho = synth.droplet_densities(192, 96, 80, 16.0, study.RHO_IN_STUDY, study.RHO_OUT_STUDY,
                                          configs.NOISE, seed=2)
        else:
            p, rho, _ = configs.config2(ca)
        s = lbfe.Solver(p)
        s.init(0, rho)
        tmp = a.out + ".part"
        open(tmp, "w").close()
        rows = run_logged(s, 0, a.steps, a.every, tmp)
        s.close()
        with open(a.out, "a") as fh:
            for r in rows:
                fh.write(json.dumps(dict(Ca=ca, **r)) + "\n")
        last = rows[-1]
        print(json.dumps({"Ca": ca, "G": p.G, "steps": last["step"], "t_over_tem": last["t_over_tem"], "D": last["D"],
                          "theta_deg": last["theta_deg"], "broken": last["broken"]}))
    import os
    os.remove(a.out + ".part")


if __name__ == "__main__":
    main()
