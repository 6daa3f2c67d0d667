"""The FP64 branch of the Peterlin factor (Eq. 2) against the FP64 oracle.

f = (L^2 - 3)/(L^2 - tr C) loses its digits to cancellation when tr C
comes close to L^2; the step kernels evaluate it in FP64 once
L^2 - tr C < 1e-2 L^2.  Here a fluid at rest carries a conformation with
tr C in [0.990, 0.999] L^2 on half of its cells (the FP64 branch) and
below that on the others; after 1 and 5 steps the GPU's C and populations
stay within 2e-6 of the oracle.  The same first step taken with the
Peterlin factor in FP32 arithmetic (computed here on the host for the
relaxation term, the only term that matters at rest) misses the oracle by
far more, which shows that the branch is what keeps the step accurate.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests.helpers import norm_err

pytestmark = pytest.mark.gpu

TOL = 2e-6


@pytest.fixture(scope="module")
def L():
    from paper_1411_2181_gb300 import build
    build.build()
    from paper_1411_2181_gb300 import lbfe
    return lbfe


def near_limit_conformation(shape, L2, seed):
    """SPD C per cell with tr C / L^2 in [0.990, 0.999] on a random half of
    the cells (checkerboard-free mix) and in [0.5, 0.98] elsewhere."""
    Lx, Ly, Lz = shape
    rng = np.random.default_rng(seed)
    n = Lx * Ly * Lz
    A = rng.uniform(-0.15, 0.15, (n, 3, 3))
    A = A + A.transpose(0, 2, 1)
    M = np.eye(3)[None] + A @ A.transpose(0, 2, 1) * 0.5 + 0.05 * A
    M = 0.5 * (M + M.transpose(0, 2, 1))
    near = rng.uniform(0, 1, n) < 0.5
    frac = np.where(near, rng.uniform(0.990, 0.999, n), rng.uniform(0.5, 0.98, n))
    M *= (frac * L2 / np.trace(M, axis1=1, axis2=2))[:, None, None]
    C = np.stack([M[:, 0, 0], M[:, 1, 1], M[:, 2, 2], M[:, 0, 1], M[:, 0, 2], M[:, 1, 2]])
    C = C.astype(np.float32)
    # the FP32 values the GPU holds must still be below the limit
    tr = C[0].astype(np.float64) + C[1] + C[2]
    assert tr.max() < L2
    return C.reshape((6, Lz, Ly, Lx)), near.reshape((Lz, Ly, Lx))


def fp32_peterlin_relaxation_step(C, L2, tau_P):
    """C after one step of the relaxation term alone, -(f C - I)/tau_P, with
    f evaluated entirely in FP32 (no FP64 branch)."""
    c = C.astype(np.float32)
    L2f = np.float32(L2)
    tr = (c[0] + c[1]) + c[2]
    f = (L2f - np.float32(3.0)) / (L2f - tr)
    delta = np.array([1, 1, 1, 0, 0, 0], np.float32).reshape((6,) + (1,) * (c.ndim - 1))
    return (c + (-(f * c - delta) * np.float32(1.0 / tau_P))).astype(np.float64)


KERNELS = [(0, 8), (0, 12), (0, 16), (1, 16)]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("L2,tau_P", [(40.0, 2000.0), (100.0, 5000.0)])
def test_peterlin_fp64_branch_matches_oracle(L, kernel, L2, tau_P):
    shape = (36, 20, 10)
    Lx, Ly, Lz = shape
    # droplet-viscoelastic fluid at rest (uniform composition, still walls);
    # a tiny polymer viscosity keeps the stress-driven flow, and with it the
    # stretching term, negligible against the relaxation under test
    p = L.Params(Lx=Lx, Ly=Ly, Lz=Lz, R=3.0, Uw=0.0, G=3.1, eta_M=0.5, eta_P=1e-8, tau_P=tau_P, L2=L2,
                 visco_phase=1)
    rho = np.empty((2, Lz, Ly, Lx))
    rho[0] = 1.0
    rho[1] = 0.04
    C0, near = near_limit_conformation(shape, L2, seed=int(L2) + kernel[1])
    s = L.Solver(p)
    s.tune(kernel[1], 0, kernel[0])
    s.init(0, rho)
    s.set_field(0, L.FIELD_C, C0)
    orc = O.Oracle(p.oracle_dict())
    orc.f[:] = s.get_field(0, L.FIELD_F)
    orc.C[:] = s.get_field(0, L.FIELD_C)
    C_start = orc.C.copy()
    s.step(1)
    orc.step(1)
    Cg = s.get_field(0, L.FIELD_C)
    e1 = norm_err(Cg, orc.C, 1)
    assert e1 < TOL, e1
    assert norm_err(s.get_field(0, L.FIELD_F), orc.f, 2) < TOL
    # the FP32-only Peterlin factor misses the oracle on the near-limit cells
    c32 = fp32_peterlin_relaxation_step(C_start, L2, tau_P)
    diff = np.abs(c32 - orc.C)[:, near].max(axis=1) / np.abs(orc.C).reshape(6, -1).max(axis=1)
    assert diff.max() > 5 * TOL, diff
    # and on the same cells the GPU does not
    diff_gpu = np.abs(Cg.astype(np.float64) - orc.C)[:, near].max(axis=1) / np.abs(orc.C).reshape(6, -1).max(axis=1)
    assert diff_gpu.max() < TOL
    s.step(4)
    orc.step(4)
    assert norm_err(s.get_field(0, L.FIELD_C), orc.C, 1) < TOL
    assert norm_err(s.get_field(0, L.FIELD_F), orc.f, 2) < TOL
    assert s.check() == L.OK
