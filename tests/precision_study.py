"""Errors of the reduced storage forms against the FP64 oracle over a long
run (test infrastructure: it runs the oracle).

The 64^3 reduced run of the strongly confined viscoelastic-droplet workload
(R = 22, W = 64, lambda = 3, De = 2, L^2 = 400) is advanced for --steps
steps by the CUDA path in FP32, FP16- and BF16-offset storage and by the
FP64 oracle, with the observables every --every steps; the script prints,
per storage form, the largest differences from the oracle in D, theta and
each component's mass, as one JSON document.  With --full-steps N the full
256 x 128 x 64 lattice of the same workload (beyond the oracle's reach in
a few minutes) is also advanced N steps in the three forms, and the reduced
forms are compared with FP32 storage.

    python -m tests.precision_study --steps 10000 --every 500 --full-steps 10000 --out precision.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--every", type=int, default=500)
    ap.add_argument("--full-steps", type=int, default=0)
    ap.add_argument("--mass-drift", action="store_true",
                    help="component masses of the reduced forms against FP32 storage every 1000 steps "
                         "over 10^4 steps on 64 x 64, 128 x 64 and 256 x 128 cross-sections")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    from paper_1411_2181_gb300 import build
    build.build()
    rep = {}
    if a.steps > 0:
        rep = crop_against_oracle(a.steps, a.every)
    if a.full_steps > 0:
        rep["full"] = full_lattice(a.full_steps, a.every)
    if a.mass_drift:
        rep["mass_drift"] = mass_drift()
    txt = json.dumps(rep, indent=1)
    print(txt)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(txt)


def crop_against_oracle(steps: int, every: int) -> dict:
    """The 64^3 crop in the three storage forms against the FP64 oracle."""
    from dataclasses import replace

    import numpy as np

    from oracle import oracle as O
    from paper_1411_2181_gb300 import configs, lbfe
    p, rho, _ = configs.config3(crop=True)
    traj = {}
    for prec in (0, 1, 2):
        s = lbfe.Solver(replace(p, precision=prec))
        s.init(0, rho)
        out = [s.observables(0)]
        for _ in range(steps // every):
            s.step(every)
            out.append(s.observables(0))
        traj[prec] = out
        s.close()
    t0 = time.time()
    o = O.Oracle(p.oracle_dict(), rho)
    ref = [o.observables()]
    for _ in range(steps // every):
        o.step(every)
        ref.append(o.observables())
    oracle_s = time.time() - t0
    rep = {"workload": "droplet_ve 64^3 crop (R 22, W 64, lambda 3, De 2, L2 400)", "steps": steps,
           "every": every, "oracle_seconds": oracle_s, "final_oracle": {"D": ref[-1]["D"],
                                                                         "theta_deg": ref[-1]["theta_deg"]}}
    for prec, name in ((0, "fp32"), (1, "fp16"), (2, "bf16")):
        g = traj[prec]
        rep[name] = {
            "max_abs_dD": max(abs(x["D"] - y["D"]) for x, y in zip(g, ref)),
            "max_abs_dtheta_deg": max(abs(x["theta_deg"] - y["theta_deg"]) for x, y in zip(g[1:], ref[1:])),
            "max_rel_mass_error": max(float((np.abs(np.array(x["mass"]) - np.array(y["mass"])) /
                                             np.array(y["mass"])).max()) for x, y in zip(g, ref)),
            "final_D": g[-1]["D"], "final_theta_deg": g[-1]["theta_deg"]}
    return rep


def full_lattice(steps: int, every: int) -> dict:
    """The full 256 x 128 x 64 lattice in the three storage forms; the
    reduced forms' largest differences from FP32 storage over the run."""
    from dataclasses import replace

    import numpy as np

    from paper_1411_2181_gb300 import configs, lbfe
    p, rho, _ = configs.config3()
    traj = {}
    t0 = time.time()
    for prec in (0, 1, 2):
        s = lbfe.Solver(replace(p, precision=prec))
        s.init(0, rho)
        out = [s.observables(0)]
        for _ in range(steps // every):
            s.step(every)
            out.append(s.observables(0))
        traj[prec] = (out, s.check())
        s.close()
    rep = {"lattice": [p.Lx, p.Ly, p.Lz], "steps": steps, "every": every, "seconds": time.time() - t0,
           "final_fp32": {"D": traj[0][0][-1]["D"], "theta_deg": traj[0][0][-1]["theta_deg"]},
           "status": {n: traj[k][1] for k, n in ((0, "fp32"), (1, "fp16"), (2, "bf16"))}}
    ref = traj[0][0]
    for prec, name in ((1, "fp16"), (2, "bf16")):
        g = traj[prec][0]
        rep[name + "_vs_fp32"] = {
            "max_abs_dD": max(abs(x["D"] - y["D"]) for x, y in zip(g, ref)),
            "max_abs_dtheta_deg": max(abs(x["theta_deg"] - y["theta_deg"]) for x, y in zip(g[1:], ref[1:])),
            "max_rel_mass_error": max(float((np.abs(np.array(x["mass"]) - np.array(y["mass"])) /
                                             np.array(y["mass"])).max()) for x, y in zip(g, ref)),
            "final_D": g[-1]["D"], "final_theta_deg": g[-1]["theta_deg"]}
    return rep


def mass_drift() -> dict:
    """The reduced forms' component masses against FP32 storage every 1000
    steps over 10^4 steps, for the same droplet and gap on three x-y
    cross-sections (absolute differences per component, and relative ones
    at the end)."""
    from dataclasses import replace

    import numpy as np

    from paper_1411_2181_gb300 import configs, lbfe, synth
    out = {}
    for Lx, Ly in ((64, 64), (128, 64), (256, 128)):
        p0, _, _ = configs.config3()
        p0 = replace(p0, Lx=Lx, Ly=Ly)
        rho = synth.droplet_densities(Lx, Ly, 64, 22.0, configs.RHO_IN, configs.RHO_OUT, configs.NOISE, seed=3)
        tr = {}
        for prec in (0, 1, 2):
            s = lbfe.Solver(replace(p0, precision=prec))
            s.init(0, rho)
            m = [s.observables(0)["mass"]]
            for _ in range(10):
                s.step(1000)
                m.append(s.observables(0)["mass"])
            tr[prec] = np.array(m)
            s.close()
        rep = {}
        for prec in (1, 2):
            d = tr[prec] - tr[0]
            rep[["", "fp16", "bf16"][prec]] = {
                "abs_A": d[:, 0].tolist(), "abs_B": d[:, 1].tolist(),
                "rel_A_end": float(d[-1, 0] / tr[0][-1, 0]), "rel_B_end": float(d[-1, 1] / tr[0][-1, 1])}
        rep["mass_fp32"] = tr[0][[0, -1]].tolist()
        out[f"{Lx}x{Ly}"] = rep
    return out


if __name__ == "__main__":
    main()
