"""Writes ``shan_chen_constants.txt``: the Shan-Chen coexistence densities
and interfacial tensions that the workloads use to convert the paper's
dimensionless groups (Ca of Sec. 1, De of Eq. 8, tau_em of Eq. 9) into
lattice parameters.  The paper does not print them (they belong to the
lattice model, not to the physics it studies); they are measured here with
the FP64 CPU oracle only:

  slab     a flat layer of component A (24 of 48 planes, 48 x 1 x 4 box)
           relaxed at rest; the bulk densities at the layer centre (majority)
           and far from it (minority);
  laplace  static cylinders along y in a 56 x 1 x 56 box, relaxed at rest;
           p = (rho_A + rho_B)/3 + G rho_A rho_B / 3 (the Shan-Chen pressure)
           inside minus outside, fitted to sigma / R + c by least squares.

Run ``python tests/golden/make_shan_chen_constants.py`` from the repository
root to regenerate the file (about a minute on one core)."""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O            # noqa: E402
from paper_1411_2181_gb300 import synth   # noqa: E402

OUT = os.path.join(HERE, "shan_chen_constants.txt")

# (name, G, initial majority, initial minority, steps)
SLABS = [("slab_G3.8", 3.8, 1.0, 0.02, 4000)]
# (name, G, rho_in, rho_out, radii, steps)
LAPLACE = [("laplace_G3.1", 3.1, 1.0, 0.04, (8, 10, 12, 14, 16), 6000),
           ("laplace_G3.8", 3.8, 1.05503, 0.01288, (10, 13, 16), 6000)]


def slab(G, a, b, steps, L=48):
    p = dict(Lx=L, Ly=1, Lz=4, Uw=0.0, G=G, eta_M=1.04 / 6, rho_in=a, rho_out=b)
    o = O.Oracle(p, synth.slab_densities(L, 1, 4, 24, rho_in=a, rho_out=b))
    o.step(steps)
    r = o.detail()["rho"][:, 1, 0, :]
    return float(r[0, L // 2]), float(r[0, 2])


def laplace(G, a, b, radii, steps, L=56):
    dp = []
    for R in radii:
        p = dict(Lx=L, Ly=1, Lz=L, Uw=0.0, G=G, eta_M=(a + b) / 6, rho_in=a, rho_out=b)
        o = O.Oracle(p, synth.cylinder_densities(L, 1, L, R, rho_in=a, rho_out=b))
        o.step(steps)
        r = o.detail()["rho"]
        P = (r[0] + r[1]) / 3 + G / 3 * r[0] * r[1]
        c = L // 2
        dp.append(P[c, 0, c] - P[c, 0, 2])
    R = np.asarray(radii, float)
    dp = np.asarray(dp)
    A = np.vstack([1 / R, np.ones_like(R)]).T
    (sigma, icpt), *_ = np.linalg.lstsq(A, dp, rcond=None)
    pred = A @ [sigma, icpt]
    r2 = 1 - ((dp - pred) ** 2).sum() / ((dp - dp.mean()) ** 2).sum()
    return float(sigma), float(icpt), float(r2), float(dp.max())


def main():
    lines = ["# Shan-Chen constants measured with the FP64 oracle; written by",
             "# make_shan_chen_constants.py (recipes in its docstring).",
             "# slab    <name> G rho_init_major rho_init_minor steps rho_major rho_minor",
             "# laplace <name> G rho_in rho_out steps radii sigma intercept R2 max_dp"]
    for name, G, a, b, steps in SLABS:
        hi, lo = slab(G, a, b, steps)
        lines.append(f"slab {name} {G} {a} {b} {steps} {hi:.5f} {lo:.5f}")
    for name, G, a, b, radii, steps in LAPLACE:
        s, c, r2, mx = laplace(G, a, b, radii, steps)
        rr = ",".join(str(r) for r in radii)
        lines.append(f"laplace {name} {G} {a} {b} {steps} {rr} {s:.5f} {c:.3e} {r2:.6f} {mx:.5f}")
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
