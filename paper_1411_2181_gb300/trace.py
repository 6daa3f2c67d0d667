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
