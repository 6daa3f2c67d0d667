"""Named workloads and the mapping from the paper's dimensionless groups to
lattice parameters.

Dimensionless groups (Sec. 1 and Sec. 2):
  Ca     = eta_M gamma_dot R / sigma, gamma_dot = 2 Uw / W      (Sec. 1, Sec. 3)
  tau_em = R eta_M / sigma                                      (Eq. 9)
  De     = (tau_P / tau_em)(eta_P / eta_M)                      (Eq. 8)
The viscoelastic phase holds a polymer fraction beta of its total viscosity:
DV: eta_P = beta lambda eta_M (eta_P/eta_d = beta); MV: eta_P = beta eta_M.

SIGMA is the interfacial tension of the Shan-Chen coupling G = 3.1 with
rho_in = 1, rho_out = 0.04, fitted from the Laplace law p_in - p_out = sigma/R
of static cylindrical droplets (R = 8..16) in the CPU oracle (recipe and
value recorded in tests/golden/shan_chen_constants.txt).  It only enters
the bookkeeping of Ca, De and tau_em.
"""
from __future__ import annotations

import math
from dataclasses import replace

import numpy as np

from . import synth

G_DEFAULT = 3.1
SIGMA = 0.0592
RHO_IN, RHO_OUT = 1.0, 0.04
NOISE = 1e-4


def make_params(Lx, Ly, Lz, R, Ca, De, lam=1.0, beta=0.4, L2=100.0, phase=1, Uw=None,
                Uw_max=0.05, G=G_DEFAULT, sigma=SIGMA, precision=0, rho_in=RHO_IN, rho_out=RHO_OUT):
    """Lattice parameters for a droplet of radius R between walls at gap
    W = Lz at capillary number Ca and Deborah number De (Eq. 8).

    With Uw given, eta_M follows from Ca; otherwise Uw = Uw_max."""
    from .params import Params
    W = Lz
    if Uw is None:
        Uw = Uw_max
    gdot = 2.0 * Uw / W
    eta_M = Ca * sigma / (gdot * R)
    if phase == 1:
        eta_P = beta * lam * eta_M
    elif phase == 2:
        eta_P = beta * eta_M
    else:
        eta_P = 0.0
    tau_em = R * eta_M / sigma
    if De > 0 and eta_P > 0:
        tau_P = De * tau_em * eta_M / eta_P
    else:
        tau_P = 1.0
        eta_P = 0.0 if De <= 0 else eta_P
        if De <= 0:
            phase = 0
    return Params(Lx=Lx, Ly=Ly, Lz=Lz, R=R, Uw=Uw, G=G, eta_M=eta_M, lambda_=lam, eta_P=eta_P,
                  tau_P=tau_P, L2=L2, visco_phase=phase, rho_in=rho_in, rho_out=rho_out,
                  sigma=sigma, precision=precision, rho0=(rho_out, rho_out))


def config1():
    """32^3 box, walls at the outer layers (W = 32) moving at -/+ 0.005,
    droplet R = 8 with a seeded centre offset, lambda = 1, viscoelastic
    droplet De = 1, L^2 = 100, eta_P/eta_d = 0.4, Ca = 0.1; 500 steps."""
    p = make_params(32, 32, 32, 8.0, Ca=0.1, De=1.0, lam=1.0, beta=0.4, L2=100.0, phase=1, Uw=0.005)
    rho = synth.droplet_densities(32, 32, 32, 8.0, RHO_IN, RHO_OUT, NOISE, seed=1)
    return p, rho, 500


def config2(Ca=0.2):
    """192 x 96 x 80, W = 80, R = 16 (2R/W = 0.4), lambda = 1, viscoelastic
    matrix De = 1, L^2 = 100, eta_P/eta_M = 0.4; Ca in {0.1, 0.2, 0.3}."""
    p = make_params(192, 96, 80, 16.0, Ca=Ca, De=1.0, lam=1.0, beta=0.4, L2=100.0, phase=2, Uw=0.02)
    rho = synth.droplet_densities(192, 96, 80, 16.0, RHO_IN, RHO_OUT, NOISE, seed=2)
    return p, rho, 20000


def config3(precision=0, crop=False):
    """256 x 128 x 64, W = 64, R = 22 (2R/W ~ 0.7), lambda = 3, viscoelastic
    droplet De = 2, L^2 = 400.  ``crop`` gives the 64^3 reduced run with the
    same W, R and parameters."""
    Lx, Ly = (64, 64) if crop else (256, 128)
    p = make_params(Lx, Ly, 64, 22.0, Ca=0.2, De=2.0, lam=3.0, beta=0.4, L2=400.0, phase=1, Uw=0.02,
                    precision=precision)
    rho = synth.droplet_densities(Lx, Ly, 64, 22.0, RHO_IN, RHO_OUT, NOISE, seed=3)
    return p, rho, 10000


def config4(n=64, seed=4):
    """Uneven batch: Lx ~ U[96, 256] (multiple of 8), Ly = Lx/2,
    W ~ U[40, 96], 2R/W ~ U[0.35, 0.75], Ca ~ U[0.05, 0.45],
    De in {0, 0.5, 1, 2}, lambda in {0.5, 1, 3}, phase DV or MV.  Draws that
    would not fit the droplet in the box (2R + 8 > Ly or 4R > Lx) are
    redrawn."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        Lx = int(rng.integers(12, 33)) * 8
        Ly = Lx // 2
        W = int(rng.integers(40, 97))
        conf = rng.uniform(0.35, 0.75)
        R = 0.5 * W * conf
        Ca = rng.uniform(0.05, 0.45)
        De = float(rng.choice([0.0, 0.5, 1.0, 2.0]))
        lam = float(rng.choice([0.5, 1.0, 3.0]))
        phase = int(rng.choice([1, 2]))
        s = int(rng.integers(0, 2 ** 31))
        if 2 * R + 8 > Ly or 4 * R > Lx:
            continue
        p = make_params(Lx, Ly, W, R, Ca=Ca, De=De, lam=lam, beta=0.4, L2=100.0, phase=phase, Uw=0.02)
        out.append((p, s))
    return out


def config4_densities(p, s):
    return synth.droplet_densities(p.Lx, p.Ly, p.Lz, p.R, RHO_IN, RHO_OUT, NOISE, seed=s)
