"""Failure path of the step kernel: a TMA copy whose completion never comes.
The test hook rebuilds the population tensor maps one row short of what the
kernel expects, so that the completion barrier of each block's first copy
stays pending; the bounded wait expires (after about a second of GPU time),
the block stops, and the host reads LBFE_ERR_TIMEOUT.  The context stays
usable: a new solver on it steps and matches the oracle."""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_1411_2181_gb300 import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1411_2181_gb300 import build
    build.build()
    from paper_1411_2181_gb300 import lbfe
    return lbfe


@pytest.mark.parametrize("kernel,ty", [(0, 8), (0, 16), (1, 16)])
def test_expired_copy_wait_reports_timeout(L, kernel, ty):
    p, rho, _ = configs.config1()          # 32^3: rows of 128 bytes, staged by TMA
    s = L.Solver(p)
    s.tune(ty, 0, kernel)
    s.init(0, rho)
    s.test_inject(L.INJECT_SHORT_COPIES)
    t0 = time.time()
    s.step(1)
    st = s.check()
    dt = time.time() - t0
    s.test_inject(0)
    s.close()
    assert st == L.ERR_TIMEOUT
    assert dt < 30.0

    s = L.Solver(p)
    s.tune(ty, 0, kernel)
    s.init(0, rho)
    s.step(3)
    assert s.check() == L.OK
    f = s.get_field(0, L.FIELD_F)
    s.close()
    o = O.Oracle(p.oracle_dict(), rho)
    o.step(3)
    assert np.abs(f - o.f).max() <= 1e-5 * np.abs(o.f).max()
