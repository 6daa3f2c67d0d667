"""The x-split domain decomposition on the GPU: slabs held by one process
(one solver each, ghost columns exchanged through the C ABI's column
blocks) advance exactly as the undivided lattice, bit for bit, in FP32 and
with FP16 storage.  The multi-GPU transport (NCCL between ranks) is the
same exchange over torch.distributed; it is covered on the CPU with gloo
ranks (tests/test_decomp.py)."""
from dataclasses import replace

import numpy as np
import pytest

from paper_1411_2181_gb300 import configs, decomp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1411_2181_gb300 import build
    build.build()
    from paper_1411_2181_gb300 import lbfe
    return lbfe


@pytest.mark.parametrize("parts", [2, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_slabs_equal_the_undivided_lattice(L, parts, prec):
    p, rho, _ = configs.config1()
    p = replace(p, precision=prec)
    steps = 30
    whole = L.Solver(p)
    whole.init(0, rho)
    whole.step(steps)
    slabs = []
    for x0, nx in decomp.partition(p.Lx, parts):
        s = L.Solver(decomp.local_params(p, nx))
        s.init(0, decomp.slab_field(rho, x0, nx))
        slabs.append(decomp.Slab(x0, nx, decomp.CudaSlabStepper(s)))
    decomp.run(slabs, decomp.LocalRing(slabs), steps)
    f = np.concatenate([decomp.interior(s.stepper.s.get_field(0, L.FIELD_F)) for s in slabs], axis=-1)
    C = np.concatenate([decomp.interior(s.stepper.s.get_field(0, L.FIELD_C)) for s in slabs], axis=-1)
    assert np.array_equal(f, whole.get_field(0, L.FIELD_F))
    assert np.array_equal(C, whole.get_field(0, L.FIELD_C))
    for s in slabs:
        assert s.stepper.s.check() == L.OK


def test_column_blocks_round_trip(L):
    p, rho, _ = configs.config1()
    s = L.Solver(replace(p, precision=1))
    s.init(0, rho)
    s.step(3)
    import torch
    n = s.columns_bytes(0, 5)
    assert n == 5 * p.Ly * p.Lz * (38 * 2 + 6 * 4 + 8)
    t = torch.empty(n, dtype=torch.uint8, device="cuda")
    f0 = s.get_field(0, L.FIELD_F)
    s.get_columns(0, 7, 5, t.data_ptr())
    s.set_columns(0, 20, 5, t.data_ptr())
    f1 = s.get_field(0, L.FIELD_F)
    assert np.array_equal(f1[..., 20:25], f0[..., 7:12])
    assert np.array_equal(np.delete(f1, range(20, 25), axis=-1), np.delete(f0, range(20, 25), axis=-1))
    with pytest.raises(L.LbfeError):
        s.get_columns(0, p.Lx - 2, 5, t.data_ptr())
