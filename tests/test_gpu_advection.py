"""The second-order minmod-limited upwind scheme for u . grad C
(advection = 1) on the GPU against the FP64 oracle's same scheme: a 500-step
droplet run, ragged random states, z-chunk boundaries (where the kernel
carries the own column's C of plane r - 2 across planes), and the reduced
storage forms."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import oracle as O
from paper_1411_2181_gb300 import configs
from tests.helpers import norm_err, random_populations, tensor_err

pytestmark = pytest.mark.gpu

TOL_500 = 1e-5
TOL_FEW = 2e-6


@pytest.fixture(scope="module")
def L():
    from paper_1411_2181_gb300 import build
    build.build()
    from paper_1411_2181_gb300 import lbfe
    return lbfe


def run_pair(L, p, rho, steps, f0=None, C0=None, z_chunk=0):
    s = L.Solver(p)
    if z_chunk:
        s.tune(8, z_chunk, 0)
    orc = O.Oracle(p.oracle_dict())
    if rho is None:
        rho = np.ones((2, p.Lz, p.Ly, p.Lx))
    s.init(0, rho)
    orc.init(rho)
    if f0 is not None:
        s.set_field(0, L.FIELD_F, f0)
    if C0 is not None:
        s.set_field(0, L.FIELD_C, C0)
    orc.f[:] = s.get_field(0, L.FIELD_F)
    orc.C[:] = s.get_field(0, L.FIELD_C)
    s.step(steps)
    orc.step(steps)
    return s, orc


def test_config1_500_steps(L):
    p, rho, steps = configs.config1()
    p = replace(p, advection=1)
    s, orc = run_pair(L, p, rho, steps)
    ef = norm_err(s.get_field(0, L.FIELD_F), orc.f, 2)
    eC = tensor_err(s.get_field(0, L.FIELD_C), orc.C)
    print(f"second-order advection, config1 500 steps: f {ef:.3e}, C {eC:.3e}")
    assert ef < TOL_500 and eC < TOL_500
    assert s.check() == L.OK


@pytest.mark.parametrize("shape", [(7, 5, 6), (33, 17, 11), (66, 19, 7), (2, 1, 2), (36, 10, 5)])
@pytest.mark.parametrize("phase", [1, 2])
def test_random_state_ragged(L, shape, phase):
    Lx, Ly, Lz = shape
    p = L.Params(Lx=Lx, Ly=Ly, Lz=Lz, R=2.0, Uw=0.03, G=3.1, eta_M=0.4, lambda_=1.3, eta_P=0.15,
                 tau_P=6.0, L2=40.0, visco_phase=phase, g=(1e-4, -3e-5, 2e-5), advection=1)
    f0, C0 = random_populations(shape, seed=3 * sum(shape) + phase)
    s, orc = run_pair(L, p, None, 1, f0, C0)
    assert norm_err(s.get_field(0, L.FIELD_F), orc.f, 2) < TOL_FEW
    assert tensor_err(s.get_field(0, L.FIELD_C), orc.C) < TOL_FEW
    s.step(4)
    orc.step(4)
    assert tensor_err(s.get_field(0, L.FIELD_C), orc.C) < 5 * TOL_FEW


@pytest.mark.parametrize("z_chunk", [3, 5, 8])
def test_z_chunk_boundaries(L, z_chunk):
    """Items start at every z-chunk boundary; the C of plane r - 2 that the
    scheme needs there comes from the item's first stage-M plane."""
    shape = (40, 20, 13)
    p = L.Params(Lx=40, Ly=20, Lz=13, R=3.0, Uw=0.03, G=3.1, eta_M=0.5, eta_P=0.2, tau_P=9.0,
                 L2=60.0, visco_phase=1, advection=1)
    f0, C0 = random_populations(shape, seed=77)
    s, orc = run_pair(L, p, None, 3, f0, C0, z_chunk=z_chunk)
    assert s.launch_config()["z_chunk"] == z_chunk
    assert tensor_err(s.get_field(0, L.FIELD_C), orc.C) < TOL_FEW
    assert norm_err(s.get_field(0, L.FIELD_F), orc.f, 2) < TOL_FEW


def test_scheme_is_active_and_shape_rules(L):
    p, rho, _ = configs.config1()
    out = {}
    for adv in (0, 1):
        s = L.Solver(replace(p, advection=adv))
        s.init(0, rho)
        s.step(50)
        out[adv] = s.get_field(0, L.FIELD_C)
        if adv:
            assert s.launch_config()["tile_y"] == 8
            for ty, kern in ((12, 0), (16, 0), (16, 1)):
                with pytest.raises(L.LbfeError) as ei:
                    s.tune(ty, 0, kern)
                assert ei.value.status == L.ERR_BAD_PARAM
        s.close()
    assert np.abs(out[1] - out[0]).max() > 1e-7


@pytest.mark.parametrize("prec", [1, 2])
def test_reduced_storage_with_second_order_advection(L, prec):
    p0, rho, _ = configs.config3(crop=True)
    out = []
    for pr in (0, prec):
        s = L.Solver(replace(p0, precision=pr, advection=1))
        s.init(0, rho)
        s.step(40)
        out.append(s.get_field(0, L.FIELD_F))
        s.close()
    scale = np.abs(out[0]).max()
    assert np.abs(out[1] - out[0]).max() <= (2e-3 if prec == 1 else 2e-2) * scale
