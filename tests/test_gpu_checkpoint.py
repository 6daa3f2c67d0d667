"""Checkpoint / resume through the C ABI (lbfe_save, lbfe_load): a run saved
after n1 steps and resumed in a new solver for n2 more steps ends bitwise
equal to the uninterrupted run, in FP32 and in the reduced storage forms
(whose offset densities travel with the file); corrupt or mismatched files
are refused."""
import os
from dataclasses import replace

import numpy as np
import pytest

from paper_1411_2181_gb300 import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1411_2181_gb300 import build
    build.build()
    from paper_1411_2181_gb300 import lbfe
    return lbfe


def state(L, s):
    return s.get_field(0, L.FIELD_F), s.get_field(0, L.FIELD_C), s.observables(0)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_resume_is_bitwise_identical(L, prec, tmp_path):
    p0, rho, _ = configs.config1()
    p = replace(p0, precision=prec)
    path = str(tmp_path / "ckpt.bin")
    a = L.Solver(p)
    a.init(0, rho)
    a.step(37)
    a.save(0, path)
    a.step(25)
    fa, Ca, oa = state(L, a)
    a.close()

    b = L.Solver(p)
    b.load(0, path)
    b.step(25)
    fb, Cb, ob = state(L, b)
    b.close()
    assert np.array_equal(fa, fb) and np.array_equal(Ca, Cb)
    assert oa["D"] == ob["D"] and oa["mass"] == ob["mass"]


def test_corrupt_or_mismatched_files_are_refused(L, tmp_path):
    p, rho, _ = configs.config1()
    path = str(tmp_path / "ckpt.bin")
    s = L.Solver(p)
    s.init(0, rho)
    s.step(3)
    s.save(0, path)
    f0 = s.get_field(0, L.FIELD_F)
    raw = bytearray(open(path, "rb").read())

    # one flipped payload byte: CRC mismatch, and the instance keeps its state
    bad = bytearray(raw)
    bad[-100] ^= 0x01
    open(path + ".bad", "wb").write(bad)
    with pytest.raises(L.LbfeError) as ei:
        s.load(0, path + ".bad")
    assert ei.value.status == L.ERR_IO
    assert np.array_equal(s.get_field(0, L.FIELD_F), f0)

    # truncated file, missing file
    open(path + ".short", "wb").write(raw[: len(raw) // 2])
    for fn in (path + ".short", str(tmp_path / "missing.bin")):
        with pytest.raises(L.LbfeError) as ei:
            s.load(0, fn)
        assert ei.value.status == L.ERR_IO
    s.close()

    # a solver with another parameter set refuses the file
    t = L.Solver(replace(p, Uw=p.Uw * 1.5))
    with pytest.raises(L.LbfeError) as ei:
        t.load(0, path)
    assert ei.value.status == L.ERR_BAD_PARAM
    t.close()
    assert os.path.getsize(path) == len(raw)
