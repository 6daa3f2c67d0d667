"""The Shan-Chen constants the workloads use (interfacial tension and
coexistence densities, which turn the paper's Ca of Sec. 1, De of Eq. 8
and tau_em of Eq. 9 into lattice parameters) against the fixture
``tests/golden/shan_chen_constants.txt`` that the oracle-only script
``tests/golden/make_shan_chen_constants.py`` writes, and the fixture
against the bulk thermodynamics and the Laplace law it must obey."""
import math
import os

import pytest

from oracle import oracle as O
from paper_1411_2181_gb300 import configs, study, synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "shan_chen_constants.txt")


@pytest.fixture(scope="module")
def golden():
    slabs, lap = {}, {}
    with open(GOLDEN) as fh:
        for line in fh:
            w = line.split()
            if not w or w[0].startswith("#"):
                continue
            if w[0] == "slab":
                slabs[w[1]] = dict(G=float(w[2]), init=(float(w[3]), float(w[4])), steps=int(w[5]),
                                   major=float(w[6]), minor=float(w[7]))
            elif w[0] == "laplace":
                lap[w[1]] = dict(G=float(w[2]), rho=(float(w[3]), float(w[4])), steps=int(w[5]),
                                 radii=[int(r) for r in w[6].split(",")], sigma=float(w[7]),
                                 icpt=float(w[8]), r2=float(w[9]), max_dp=float(w[10]))
    return slabs, lap


def test_workload_constants_match_fixture(golden):
    slabs, lap = golden
    g31, g38, s38 = lap["laplace_G3.1"], lap["laplace_G3.8"], slabs["slab_G3.8"]
    assert configs.G_DEFAULT == g31["G"] and (configs.RHO_IN, configs.RHO_OUT) == g31["rho"]
    assert abs(configs.SIGMA - g31["sigma"]) <= 1e-4
    assert study.G_STUDY == s38["G"] == g38["G"]
    assert (study.RHO_IN_STUDY, study.RHO_OUT_STUDY) == (s38["major"], s38["minor"])
    # the tension of the study's coupling is measured at its coexistence densities
    assert g38["rho"] == (s38["major"], s38["minor"])
    assert study.SIGMA_STUDY == g38["sigma"]


def test_fixture_obeys_laplace_law(golden):
    _, lap = golden
    for v in lap.values():
        assert v["sigma"] > 0 and v["r2"] > 0.999
        assert abs(v["icpt"]) < 0.05 * v["max_dp"]
    # a stronger coupling gives a sharper, stiffer interface
    assert lap["laplace_G3.8"]["sigma"] > lap["laplace_G3.1"]["sigma"]


def test_fixture_obeys_bulk_coexistence(golden):
    """Equal bulk chemical potentials ln rho_s + G rho_t of the two
    symmetric phases give ln(a/b) = G (a - b); lattice corrections grow
    with G (4% at G = 3.1, 11% at 3.8)."""
    slabs, _ = golden
    for v in slabs.values():
        a, b = v["major"], v["minor"]
        assert a > 1.0 > b > 0
        assert abs(math.log(a / b) / (v["G"] * (a - b)) - 1) < 0.15


def test_oracle_reproduces_fixture_slab(golden):
    slabs, _ = golden
    v = slabs["slab_G3.8"]
    L = 48
    a0, b0 = v["init"]
    p = dict(Lx=L, Ly=1, Lz=4, Uw=0.0, G=v["G"], eta_M=1.04 / 6, rho_in=a0, rho_out=b0)
    o = O.Oracle(p, synth.slab_densities(L, 1, 4, 24, rho_in=a0, rho_out=b0))
    o.step(v["steps"])
    r = o.detail()["rho"][:, 1, 0, :]
    assert abs(r[0, L // 2] - v["major"]) < 1e-5 and abs(r[0, 2] - v["minor"]) < 1e-5
