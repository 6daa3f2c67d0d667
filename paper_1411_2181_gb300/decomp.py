"""Domain split along x for lattices larger than one GPU (the paper's own
runs use 1024-1356 x 128 x 128-256 cells, Sec. 3).

The lattice is cut into slabs of whole x-columns, one per rank.  Every
stencil of one time step reaches at most two cells (the Shan-Chen force and
the polymer-stress divergence at the neighbours of a cell need the moments
two columns away; streaming moves populations one column), so a slab that
holds GHOST = 2 copies of each neighbour's edge columns on either side,
refreshed before every step, advances its interior columns exactly as the
undivided periodic lattice does; what the step leaves in the ghost columns
is discarded.  One exchange per step moves, across each face, the stored
state (populations, conformation and, in the reduced forms, the offset
densities) of two columns: each slab sends its first two interior columns
to its left neighbour and its last two to its right neighbour.

The slab steppers provide four calls (the CUDA solver through the C ABI's
column blocks, ``lbfe_get_columns`` / ``lbfe_set_columns``):
  block_bytes(nx)        size of a block of nx columns (any layout);
  get_columns(x0, nx)    a 1-D tensor holding columns [x0, x0 + nx);
  set_columns(x0, nx, t) write such a tensor back;
  step(n)                advance the local lattice (periodic in x) by n steps.
Transports move the blocks: ``TorchDistTransport`` between the ranks of a
torch.distributed group (NCCL on GPUs, gloo on CPUs), ``LocalRing`` between
slabs held by one process.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

GHOST = 2


def partition(Lx: int, parts: int) -> list[tuple[int, int]]:
    """(x0, nx) of each slab: contiguous, as even as possible, nx >= GHOST."""
    if parts < 1 or Lx < GHOST * parts:
        raise ValueError(f"cannot split {Lx} columns into {parts} slabs of at least {GHOST}")
    base, extra = divmod(Lx, parts)
    out, x0 = [], 0
    for r in range(parts):
        nx = base + (1 if r < extra else 0)
        out.append((x0, nx))
        x0 += nx
    return out


def local_params(p, nx: int):
    """Parameters of a slab of nx interior columns plus the ghosts."""
    return replace(p, Lx=nx + 2 * GHOST)


def slab_field(field: np.ndarray, x0: int, nx: int) -> np.ndarray:
    """The columns x0 - GHOST .. x0 + nx + GHOST - 1 (periodic) of a field
    whose last axis is x: the slab's initial data, ghosts included."""
    Lx = field.shape[-1]
    cols = [(x0 - GHOST + i) % Lx for i in range(nx + 2 * GHOST)]
    return np.ascontiguousarray(field[..., cols])


def interior(field: np.ndarray) -> np.ndarray:
    """The interior columns of a slab field (last axis x)."""
    return field[..., GHOST:-GHOST]


class LocalRing:
    """Exchange between the slabs of one process, in slab order around the
    periodic x-direction."""

    def __init__(self, slabs: list):
        self.slabs = slabs

    def exchange(self):
        n = len(self.slabs)
        outgoing = []
        for s in self.slabs:
            outgoing.append((s.stepper.get_columns(GHOST, GHOST), s.stepper.get_columns(s.nx, GHOST)))
        for r, s in enumerate(self.slabs):
            # left ghosts <- the left neighbour's last interior columns
            s.stepper.set_columns(0, GHOST, outgoing[(r - 1) % n][1])
            # right ghosts <- the right neighbour's first interior columns
            s.stepper.set_columns(s.nx + GHOST, GHOST, outgoing[(r + 1) % n][0])


class TorchDistTransport:
    """Exchange with the neighbouring ranks of a torch.distributed group.
    Sends go right then left and receives come from the left then the
    right, so that with two ranks (both neighbours the same rank) the
    messages pair in order also on transports that ignore tags (NCCL)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def exchange_slab(self, slab):
        dist = self.dist
        s = slab.stepper
        left, right = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        send_right = s.get_columns(slab.nx, GHOST)     # my last interior columns
        send_left = s.get_columns(GHOST, GHOST)        # my first interior columns
        recv_left = send_right.new_empty(send_right.shape)
        recv_right = send_left.new_empty(send_left.shape)
        if self.world == 1:
            recv_left.copy_(send_right)
            recv_right.copy_(send_left)
        else:
            gl = dist.get_global_rank(self.group, left) if self.group is not None else left
            gr = dist.get_global_rank(self.group, right) if self.group is not None else right
            ops = [dist.P2POp(dist.isend, send_right, gr, self.group, 1),
                   dist.P2POp(dist.isend, send_left, gl, self.group, 2),
                   dist.P2POp(dist.irecv, recv_left, gl, self.group, 1),
                   dist.P2POp(dist.irecv, recv_right, gr, self.group, 2)]
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        s.set_columns(0, GHOST, recv_left)
        s.set_columns(slab.nx + GHOST, GHOST, recv_right)


class Slab:
    """One slab: its interior extent and its local stepper."""

    def __init__(self, x0: int, nx: int, stepper):
        self.x0, self.nx, self.stepper = x0, nx, stepper


def run(slabs_or_slab, transport, steps: int):
    """Advance by `steps` time steps: one ghost exchange, then one local
    step, per time step."""
    slabs = slabs_or_slab if isinstance(slabs_or_slab, list) else [slabs_or_slab]
    for _ in range(steps):
        if isinstance(transport, LocalRing):
            transport.exchange()
        else:
            for s in slabs:
                transport.exchange_slab(s)
        for s in slabs:
            s.stepper.step(1)


class CudaSlabStepper:
    """A slab on the GPU: one lbfe solver instance (its own lattice is
    periodic over the slab width, ghosts included) and device buffers for
    the column blocks."""

    def __init__(self, solver, k: int = 0):
        import torch
        self.torch = torch
        self.s, self.k = solver, k
        self.device = solver.device

    def block_bytes(self, nx: int) -> int:
        return self.s.columns_bytes(self.k, nx)

    def get_columns(self, x0: int, nx: int):
        t = self.torch.empty(self.block_bytes(nx), dtype=self.torch.uint8, device=self.device)
        self.s.get_columns(self.k, x0, nx, t.data_ptr())
        return t

    def set_columns(self, x0: int, nx: int, t):
        self.s.set_columns(self.k, x0, nx, t.data_ptr())

    def step(self, n: int):
        self.s.step(n)
