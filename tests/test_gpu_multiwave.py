"""The step kernel's multi-wave path: more work items than resident blocks.

A launch whose work items (column tile x z-chunk, over all instances)
outnumber its persistent blocks hands out the items beyond the first wave
from a counter in device memory, one item ahead (the next item's first
plane is copied while the current one runs); the last block to finish
resets the counter for the next launch.  These tests force that path and
compare it with the oracle, with single-wave runs (bit for bit: the
arithmetic of a cell does not depend on which block or item computes it)
and across consecutive launches and CUDA-graph replays (a counter left
non-zero would skip items in the next launch).
"""
from dataclasses import replace

import numpy as np
import pytest

from oracle import oracle as O
from paper_1411_2181_gb300 import configs, synth
from tests.helpers import norm_err, random_populations, tensor_err

pytestmark = pytest.mark.gpu

TOL_FEW = 2e-6


@pytest.fixture(scope="module")
def L():
    from paper_1411_2181_gb300 import build
    build.build()
    from paper_1411_2181_gb300 import lbfe
    return lbfe


@pytest.fixture(scope="module")
def cfg2_oracle():
    """Config 2 (192 x 96 x 80, matrix viscoelastic) from a perturbed state,
    and the oracle after 3 steps."""
    p, rho, _ = configs.config2(0.2)
    f0, C0 = random_populations((p.Lx, p.Ly, p.Lz), seed=21, amp=0.01)
    f0 = f0.astype(np.float32)
    C0 = C0.astype(np.float32)
    orc = O.Oracle(p.oracle_dict())
    orc.f[:] = f0
    orc.C[:] = C0
    orc.step(3)
    return p, rho, f0, C0, orc


def _solver(L, p, rho, f0, C0, tile_y, z_chunk, kernel):
    s = L.Solver(p)
    s.tune(tile_y, z_chunk, kernel)
    s.init(0, rho)
    s.set_field(0, L.FIELD_F, f0)
    s.set_field(0, L.FIELD_C, C0)
    return s


# (kernel, tile_y): one cell per thread at 8, 12 and 16 rows, two cells per thread
SHAPES = [(0, 8), (0, 12), (0, 16), (1, 16)]


@pytest.mark.parametrize("kernel,tile_y", SHAPES)
def test_config2_multiwave_matches_oracle(L, cfg2_oracle, kernel, tile_y):
    """Config 2 with 8-plane z-chunks: hundreds of items on at most one
    block per SM; 3 steps (a graph replay) against the oracle."""
    p, rho, f0, C0, orc = cfg2_oracle
    s = _solver(L, p, rho, f0, C0, tile_y, 8, kernel)
    cfg = s.launch_config()
    assert cfg["items"] > cfg["grid"], cfg
    s.step(3)
    assert norm_err(s.get_field(0, L.FIELD_F), orc.f, 2) < TOL_FEW
    assert tensor_err(s.get_field(0, L.FIELD_C), orc.C) < TOL_FEW
    assert s.check() == L.OK


@pytest.mark.parametrize("kernel,tile_y", SHAPES)
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_config2_multiwave_equals_single_wave(L, cfg2_oracle, kernel, tile_y, prec):
    """The same steps with every item in the first wave (one z-chunk per
    column tile) and with 8-plane chunks on several waves give identical
    fields, in FP32, FP16 and BF16 storage (stochastic rounding), over
    single steps and graph replays."""
    p, rho, f0, C0, _ = cfg2_oracle
    p = replace(p, precision=prec)
    one = _solver(L, p, rho, f0, C0, tile_y, p.Lz, kernel)
    many = _solver(L, p, rho, f0, C0, tile_y, 8, kernel)
    c1, cm = one.launch_config(), many.launch_config()
    assert c1["items"] <= c1["grid"] and cm["items"] > cm["grid"], (c1, cm)
    for n in (1, 2, 1, 3):
        one.step(n)
        many.step(n)
    assert np.array_equal(one.get_field(0, L.FIELD_F), many.get_field(0, L.FIELD_F))
    assert np.array_equal(one.get_field(0, L.FIELD_C), many.get_field(0, L.FIELD_C))
    assert many.check() == L.OK


def _uneven_batch(L, n=18, seed=12):
    rng = np.random.default_rng(seed)
    ps, rhos = [], []
    for k in range(n):
        Lx = int(rng.integers(3, 9)) * 8 + int(rng.integers(0, 3))   # some not multiples of 4 (no TMA)
        Ly = int(rng.integers(10, 30))
        Lz = int(rng.integers(10, 26))
        R = 0.3 * min(Lx, Ly, Lz)
        phase = int(rng.integers(0, 3))
        p = L.Params(Lx=Lx, Ly=Ly, Lz=Lz, R=R, Uw=float(rng.uniform(0.005, 0.03)), G=3.1,
                     eta_M=float(rng.uniform(0.3, 0.9)), lambda_=float(rng.choice([0.5, 1.0, 3.0])),
                     eta_P=0.1 if phase else 0.0, tau_P=float(rng.uniform(5, 40)), L2=100.0,
                     visco_phase=phase, sigma=0.0592)
        ps.append(p)
        rhos.append(synth.droplet_densities(Lx, Ly, Lz, R, seed=100 + k))
    return ps, rhos


@pytest.mark.parametrize("kernel,tile_y", SHAPES)
def test_uneven_batch_multiwave_equals_solo_runs(L, kernel, tile_y):
    """18 uneven instances with 4-plane z-chunks (several waves of items in
    one launch): after single steps and graph replays each equals its own
    solo run bit for bit; one of them matches the oracle."""
    ps, rhos = _uneven_batch(L)
    if kernel == 1:
        ps = [replace(p, Lx=p.Lx + (p.Lx % 2)) for p in ps]
        rhos = [synth.droplet_densities(p.Lx, p.Ly, p.Lz, p.R, seed=100 + k) for k, p in enumerate(ps)]
    batch = L.Solver(ps)
    batch.tune(tile_y, 4, kernel)
    cfg = batch.launch_config()
    assert cfg["items"] > cfg["grid"], cfg
    for k, r in enumerate(rhos):
        batch.init(k, r)
    schedule = (1, 3, 1, 2)
    for n in schedule:
        batch.step(n)
    assert batch.check() == L.OK
    for k, (p, r) in enumerate(zip(ps, rhos)):
        solo = L.Solver(p)
        solo.tune(tile_y, 0, kernel)
        solo.init(0, r)
        solo.step(sum(schedule))
        assert np.array_equal(batch.get_field(k, L.FIELD_F), solo.get_field(0, L.FIELD_F)), k
        assert np.array_equal(batch.get_field(k, L.FIELD_C), solo.get_field(0, L.FIELD_C)), k
        solo.close()
    k = 5
    orc = O.Oracle(ps[k].oracle_dict(), rhos[k])
    solo = L.Solver(ps[k])
    solo.init(0, rhos[k])
    orc.f[:] = solo.get_field(0, L.FIELD_F)
    orc.C[:] = solo.get_field(0, L.FIELD_C)
    orc.step(sum(schedule))
    assert norm_err(batch.get_field(k, L.FIELD_F), orc.f, 2) < 5 * TOL_FEW
    assert tensor_err(batch.get_field(k, L.FIELD_C), orc.C) < 5 * TOL_FEW


@pytest.mark.parametrize("kernel,tile_y", [(0, 8), (1, 16)])
def test_bf16_step_counts_are_per_instance(L, kernel, tile_y):
    """BF16 storage draws its rounding bits from each instance's own step
    count: a batch member re-initialised in the middle of a run restarts
    its count and equals a fresh solo run, the others equal solo runs of
    the whole schedule, bit for bit."""
    ps, rhos = _uneven_batch(L, n=3, seed=21)
    ps = [replace(p, Lx=p.Lx + (p.Lx % 2), precision=2) for p in ps]
    rhos = [synth.droplet_densities(p.Lx, p.Ly, p.Lz, p.R, seed=200 + k) for k, p in enumerate(ps)]
    batch = L.Solver(ps)
    batch.tune(tile_y, 0, kernel)
    for k, r in enumerate(rhos):
        batch.init(k, r)
    batch.step(3)
    batch.init(1, rhos[1])
    batch.step(1)
    batch.step(4)
    assert batch.check() == L.OK
    for k, (p, r) in enumerate(zip(ps, rhos)):
        solo = L.Solver(p)
        solo.tune(tile_y, 0, kernel)
        solo.init(0, r)
        solo.step(5 if k == 1 else 8)
        assert np.array_equal(batch.get_field(k, L.FIELD_F), solo.get_field(0, L.FIELD_F)), k
        solo.close()
