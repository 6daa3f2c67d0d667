"""The x-split domain decomposition on the CPU: slabs stepped by the FP64
oracle (the reference stepper of these tests) exchange their ghost columns
through torch.distributed with gloo ranks, or in one process; the assembled
interiors equal the undivided lattice's after several steps."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_1411_2181_gb300 import decomp
from paper_1411_2181_gb300.params import Params
from tests.helpers import random_populations


class OracleSlabStepper:
    """A slab stepped by the oracle; column blocks as float64 tensors."""

    def __init__(self, orc):
        self.o = orc

    def block_bytes(self, nx):
        Lz, Ly = self.o.shape[0], self.o.shape[1]
        return 8 * nx * Ly * Lz * 44

    def get_columns(self, x0, nx):
        f = self.o.f.reshape(38, *self.o.shape)[..., x0:x0 + nx]
        C = self.o.C[..., x0:x0 + nx]
        return torch.from_numpy(np.concatenate([f.ravel(), C.ravel()]))

    def set_columns(self, x0, nx, t):
        a = t.numpy()
        nf = 38 * self.o.shape[0] * self.o.shape[1] * nx
        self.o.f.reshape(38, *self.o.shape)[..., x0:x0 + nx] = a[:nf].reshape(38, *self.o.shape[:2], nx)
        self.o.C[..., x0:x0 + nx] = a[nf:].reshape(6, *self.o.shape[:2], nx)

    def step(self, n):
        self.o.step(n)


PARAMS = dict(Ly=9, Lz=7, R=2.5, Uw=0.03, G=3.1, eta_M=0.45, lambda_=1.5, eta_P=0.15, tau_P=8.0, L2=50.0,
              g=(1e-4, 2e-5, -3e-5))


def _problem(Lx, phase, seed):
    p = Params(Lx=Lx, visco_phase=phase, **PARAMS)
    f0, C0 = random_populations((Lx, p.Ly, p.Lz), seed=seed)
    return p, f0, C0


def _reference(p, f0, C0, steps):
    o = O.Oracle(p.oracle_dict())
    o.f[:] = f0
    o.C[:] = C0
    o.step(steps)
    return o.f, o.C


def _slab(p, f0, C0, x0, nx):
    lp = decomp.local_params(p, nx)
    o = O.Oracle(lp.oracle_dict())
    o.f[:] = decomp.slab_field(f0, x0, nx)
    o.C[:] = decomp.slab_field(C0, x0, nx)
    return decomp.Slab(x0, nx, OracleSlabStepper(o))


def test_partition_covers_the_lattice_once():
    for Lx, parts in ((37, 2), (37, 3), (192, 8), (8, 4)):
        sl = decomp.partition(Lx, parts)
        assert sum(nx for _, nx in sl) == Lx
        assert [x0 for x0, _ in sl] == list(np.cumsum([0] + [nx for _, nx in sl[:-1]]))
        assert max(nx for _, nx in sl) - min(nx for _, nx in sl) <= 1
        assert min(nx for _, nx in sl) >= decomp.GHOST
    with pytest.raises(ValueError):
        decomp.partition(5, 3)


def test_slab_field_wraps_periodically():
    a = np.arange(10.0)[None, :]
    s = decomp.slab_field(a, 0, 4)
    assert s.tolist() == [[8, 9, 0, 1, 2, 3, 4, 5]]
    assert decomp.interior(s).tolist() == [[0, 1, 2, 3]]


@pytest.mark.parametrize("Lx,parts,phase", [(24, 3, 1), (23, 2, 2), (20, 4, 0)])
def test_slabs_in_one_process_equal_the_undivided_lattice(Lx, parts, phase):
    p, f0, C0 = _problem(Lx, phase, seed=Lx + parts)
    steps = 4
    fr, Cr = _reference(p, f0, C0, steps)
    slabs = [_slab(p, f0, C0, x0, nx) for x0, nx in decomp.partition(Lx, parts)]
    decomp.run(slabs, decomp.LocalRing(slabs), steps)
    f = np.concatenate([decomp.interior(s.stepper.o.f) for s in slabs], axis=-1)
    C = np.concatenate([decomp.interior(s.stepper.o.C) for s in slabs], axis=-1)
    # the same FP64 arithmetic per cell: equal to the last bit
    assert np.array_equal(f, fr) and np.array_equal(C, Cr)


def test_without_the_exchange_the_slab_edges_go_wrong():
    """The exchange is what keeps the slabs exact: stepping the slabs with
    their ghosts never refreshed departs from the undivided lattice at the
    slab edges."""
    Lx, parts = 24, 2
    p, f0, C0 = _problem(Lx, 1, seed=3)
    fr, _ = _reference(p, f0, C0, 3)
    slabs = [_slab(p, f0, C0, x0, nx) for x0, nx in decomp.partition(Lx, parts)]
    for s in slabs:
        s.stepper.step(3)
    f = np.concatenate([decomp.interior(s.stepper.o.f) for s in slabs], axis=-1)
    assert np.abs(f - fr).max() > 1e-6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, Lx, phase, steps, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, f0, C0 = _problem(Lx, phase, seed=Lx * 7 + world)
    x0, nx = decomp.partition(Lx, world)[rank]
    slab = _slab(p, f0, C0, x0, nx)
    decomp.run(slab, decomp.TorchDistTransport(), steps)
    q.put((rank, x0, decomp.interior(slab.stepper.o.f).copy(), decomp.interior(slab.stepper.o.C).copy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,Lx,phase", [(2, 22, 1), (3, 25, 2)])
def test_gloo_ranks_equal_the_undivided_lattice(world, Lx, phase):
    steps = 4
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, Lx, phase, steps, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    parts = sorted((q.get(timeout=180) for _ in range(world)), key=lambda t: t[1])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p, f0, C0 = _problem(Lx, phase, seed=Lx * 7 + world)
    fr, Cr = _reference(p, f0, C0, steps)
    f = np.concatenate([t[2] for t in parts], axis=-1)
    C = np.concatenate([t[3] for t in parts], axis=-1)
    assert np.array_equal(f, fr) and np.array_equal(C, Cr)
