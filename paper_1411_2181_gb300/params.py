"""Parameters of one droplet instance, mirroring ``lbfe_params`` of
``include/lbfe.h`` (pure Python: usable without the CUDA library)."""
from __future__ import annotations

from dataclasses import dataclass

FP32, FP16_OFFSET, BF16_OFFSET = 0, 1, 2
NEWTONIAN, DROPLET_VISCOELASTIC, MATRIX_VISCOELASTIC = 0, 1, 2
ADVECTION_UPWIND1, ADVECTION_UPWIND2_MINMOD = 0, 1


@dataclass
class Params:
    """One droplet instance (lattice units); mirrors ``lbfe_params``."""
    Lx: int
    Ly: int
    Lz: int
    R: float = 8.0
    Uw: float = 0.0
    G: float = 3.1
    eta_M: float = 1.0
    lambda_: float = 1.0
    eta_P: float = 0.0
    tau_P: float = 1.0
    L2: float = 100.0
    visco_phase: int = NEWTONIAN
    rho_in: float = 1.0
    rho_out: float = 0.04
    sigma: float = 0.0
    g: tuple = (0.0, 0.0, 0.0)
    precision: int = FP32
    rho0: tuple = (0.0, 0.0)
    advection: int = ADVECTION_UPWIND1

    def oracle_dict(self) -> dict:
        """The same parameters as the plain dict the CPU oracle takes."""
        return dict(Lx=self.Lx, Ly=self.Ly, Lz=self.Lz, visco_phase=self.visco_phase, Uw=self.Uw,
                    G=self.G, eta_M=self.eta_M, **{"lambda": self.lambda_}, eta_P=self.eta_P,
                    tau_P=self.tau_P, L2=self.L2, rho_in=self.rho_in, rho_out=self.rho_out,
                    g=tuple(self.g), advection=self.advection)

    @property
    def N(self) -> int:
        return self.Lx * self.Ly * self.Lz
