"""The allocation-free observables entry point.

Callers whose device memory belongs to another allocator, or that run
under a fixed device-memory budget, cannot let the library allocate when
they ask for diagnostics; ``lbfe_observables_noalloc`` serves them from a
static device scratch array.  These checks compare it, through the C ABI,
with the handle API's ``lbfe_observables`` on the same state, twice in a
row (the shared scratch must not carry anything from one call to the
next).  The file is collected last on purpose.
"""
from dataclasses import replace

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1411_2181_gb300 import build
    build.build()
    from paper_1411_2181_gb300 import lbfe
    return lbfe


def _compare(a, b):
    for k in ("volume", "Lp", "necks", "fragments", "broken"):
        assert a[k] == b[k], k
    assert abs(a["D"] - b["D"]) < 1e-10
    assert abs(a["theta_deg"] - b["theta_deg"]) < 1e-8
    assert np.allclose(a["centroid"], b["centroid"], atol=1e-9)
    assert np.allclose(a["M"], b["M"], rtol=1e-12, atol=1e-9)
    assert np.allclose(a["mass"], b["mass"], rtol=1e-12)


def test_noalloc_matches_handle_observables_twice(L):
    import torch
    from paper_1411_2181_gb300 import configs
    p, rho, _ = configs.config1()
    s = L.Solver(p)
    s.init(0, rho)
    for steps in (150, 90):
        s.step(steps)
        ref = s.observables(0)
        f = torch.from_numpy(s.get_field(0, L.FIELD_F)).cuda()
        torch.cuda.synchronize()
        for _ in range(2):
            out = L.observables_noalloc(p, f.data_ptr(), p.N)
            _compare(out, ref)


def test_noalloc_rejects_lx_beyond_static_scratch(L):
    from paper_1411_2181_gb300 import configs
    p, _, _ = configs.config1()
    big = replace(p, Lx=4100, Ly=2, Lz=4)
    with pytest.raises(L.LbfeError) as ei:
        L.observables_noalloc(big, 1 << 20, big.N)
    assert ei.value.status == L.ERR_BAD_PARAM
