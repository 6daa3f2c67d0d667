"""The C ABI library loads and exports every symbol ``include/lbfe.h``
declares; host-side validation works without a GPU (no compute calls)."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbfe():
    from paper_1411_2181_gb300 import build
    build.build()
    from paper_1411_2181_gb300 import lbfe as L
    return L


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "lbfe.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbfe_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lbfe):
    names = declared_functions()
    assert len(names) >= 14
    lib = ct.CDLL(lbfe.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_sizes_match(lbfe):
    assert lbfe._lib.lbfe_params_size() == ct.sizeof(lbfe.CParams)
    assert lbfe._lib.lbfe_obs_size() == ct.sizeof(lbfe.CObs)


def test_parameter_validation_on_host(lbfe):
    from paper_1411_2181_gb300 import configs
    p, _, _ = configs.config1()
    d = lbfe.derive(p)
    # Sec. 1 / Eq. 9 / Eq. 8 bookkeeping
    assert abs(d["gamma_dot"] - 2 * p.Uw / p.Lz) < 1e-15
    assert abs(d["Ca"] - 0.1) < 1e-12
    assert abs(d["tau_em"] - p.R * p.eta_M / p.sigma) < 1e-9
    assert abs(d["De"] - 1.0) < 1e-12
    assert d["tau_A"] > 0.5 and d["tau_B"] > 0.5
    bad = [dict(Lz=1), dict(tau_P=0.0), dict(L2=3.0), dict(Uw=0.2), dict(eta_P=10.0),
           dict(visco_phase=5), dict(precision=9), dict(eta_M=-1.0), dict(Lx=0),
           dict(Lx=4097), dict(Lx=4096, Ly=4096, Lz=5)]
    from dataclasses import replace
    for kw in bad:
        with pytest.raises(lbfe.LbfeError) as ei:
            lbfe.derive(replace(p, **kw))
        assert ei.value.status == lbfe.ERR_BAD_PARAM, kw


def test_required_bytes_and_batch_precision_rule(lbfe):
    from dataclasses import replace
    from paper_1411_2181_gb300 import configs
    p, _, _ = configs.config1()
    n1 = lbfe.required_bytes([p])
    n2 = lbfe.required_bytes([p, p])
    assert n2 > n1 > p.N * (2 * 19 * 4 * 2 + 6 * 4 * 2)
    with pytest.raises(lbfe.LbfeError):
        lbfe.required_bytes([p, replace(p, precision=1)])
    half = lbfe.required_bytes([replace(p, precision=1)])
    assert half < n1


def test_create_rejects_small_or_misaligned_block(lbfe):
    from paper_1411_2181_gb300 import configs
    p, _, _ = configs.config1()
    arr = (lbfe.CParams * 1)(lbfe._to_c(p))
    h = ct.c_void_p()
    need = lbfe.required_bytes([p])
    # never dereferenced: both are rejected before any CUDA call
    assert lbfe._lib.lbfe_create(ct.byref(h), arr, 1, ct.c_void_p(4096), need - 1, None) == lbfe.ERR_NO_MEMORY
    assert lbfe._lib.lbfe_create(ct.byref(h), arr, 1, ct.c_void_p(4096 + 8), need, None) == lbfe.ERR_BAD_PARAM
    assert lbfe._lib.lbfe_create(ct.byref(h), arr, 0, ct.c_void_p(4096), need, None) == lbfe.ERR_BAD_PARAM


def test_test_inject_rejects_null_handle(lbfe):
    assert lbfe._lib.lbfe_test_inject(None, lbfe.INJECT_SHORT_COPIES) == lbfe.ERR_BAD_PARAM


def test_crc32_known_answers(lbfe):
    """CRC-32 check values of the reflected 0xEDB88320 polynomial: the
    standard check string, the empty input, and continuation in pieces."""
    crc = lbfe._lib.lbfe_crc32
    s = b"123456789"
    assert crc(s, len(s), 0) == 0xCBF43926
    assert crc(b"", 0, 0) == 0
    assert crc(s[4:], 5, crc(s, 4, 0)) == 0xCBF43926
    assert crc(b"a", 1, 0) == 0xE8B7BE43


def test_checkpoint_calls_reject_null_arguments(lbfe):
    assert lbfe._lib.lbfe_save(None, 0, b"/nonexistent/x") == lbfe.ERR_BAD_PARAM
    assert lbfe._lib.lbfe_load(None, 0, b"/nonexistent/x") == lbfe.ERR_BAD_PARAM


def test_deborah_number_from_n1(lbfe):
    """Eq. 5 with the steady-shear N1 of Eq. 7 (De_N1) against Eq. 8 (De):
    equal in the Oldroyd-B limit, and a few percent apart at L^2 = 100 in
    the benchmark workload (the paper's estimate of the difference)."""
    from dataclasses import replace
    from paper_1411_2181_gb300 import configs
    p, _, _ = configs.config2(0.2)
    d = lbfe.derive(p)
    assert 0.97 < d["De_N1"] / d["De"] < 1.0
    big = lbfe.derive(replace(p, L2=1e10))
    assert abs(big["De_N1"] / big["De"] - 1) < 1e-6


def test_deborah_number_from_oracle_steady_shear(lbfe):
    """De_N1 of the C ABI against N1 measured on the oracle: its FD FENE-P
    update driven by the workload's shear rate to steady state, then
    N1 = (eta_P/tau_P) f (C_xx - C_yy) in Eq. 5."""
    import numpy as np
    from oracle import oracle as O
    from paper_1411_2181_gb300 import configs
    p, _, _ = configs.config2(0.3)
    d = lbfe.derive(p)
    Lx, Ly, Lz = 1, 1, 2
    gdot = d["gamma_dot"]
    Uw = gdot * Lz / 2
    q = dict(Lx=Lx, Ly=Ly, Lz=Lz, Uw=Uw, eta_M=1, tau_P=p.tau_P, L2=p.L2)
    z = np.arange(Lz)
    u = np.zeros((3, Lz, Ly, Lx))
    u[0] = (Uw * (2 * (z + 0.5) / Lz - 1))[:, None, None]
    C = np.zeros((6, Lz, Ly, Lx))
    C[:3] = 1.0
    for _ in range(int(40 * p.tau_P)):
        C = O.fene_update(q, C, u)
    f = (p.L2 - 3) / (p.L2 - (C[0] + C[1] + C[2]))
    N1 = float((p.eta_P / p.tau_P) * (f * (C[0] - C[1])).mean())
    De_num = N1 * p.R / (2 * p.sigma * d["Ca"] ** 2)
    assert abs(De_num / d["De_N1"] - 1) < 1e-6


def test_advection_scheme_validation(lbfe):
    from dataclasses import replace
    from paper_1411_2181_gb300 import configs
    p, _, _ = configs.config1()
    assert lbfe.derive(replace(p, advection=1))["Ca"] > 0
    import pytest as _pt
    with _pt.raises(lbfe.LbfeError) as ei:
        lbfe.derive(replace(p, advection=2))
    assert ei.value.status == lbfe.ERR_BAD_PARAM
    with _pt.raises(lbfe.LbfeError) as ei:
        lbfe.required_bytes([p, replace(p, advection=1)])
    assert ei.value.status == lbfe.ERR_BAD_PARAM
