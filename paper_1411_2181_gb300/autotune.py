"""Autotuner of the step kernel's launch shape.

The step kernel runs one block per column tile and z-chunk, in one of two
variants: one cell per thread with tiles of 32 x TY cells (TY = 8, 12 or 16)
or two x-adjacent cells per thread with 32 x 16 tiles (even Lx only).  The
variant, tile height and chunk depth change speed only (the fields agree to
FP32 rounding).  ``tune`` times each candidate on a scratch solver built
from the same parameters, keeps the fastest, and caches the choice in a JSON
file keyed by the GPU name, the precision and the lattice sizes of the
batch.
"""
from __future__ import annotations

import json
import os

import numpy as np

from .params import Params

TILE_Y = (8, 12, 16)
Z_CHUNKS = (0, 8, 10, 12, 16, 20, 24, 27, 32, 40)
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _key(params: list[Params], gpu: str) -> str:
    dims = ";".join(f"{p.Lx}x{p.Ly}x{p.Lz}" for p in params)
    return f"{gpu}|v2|prec{params[0].precision}|adv{params[0].advection}|n{len(params)}|{dims}"


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def candidates(params: list[Params]):
    """(kernel, tile_y, z_chunk) triples: cell kernel (0) at every tile
    height, pair kernel (1) at 16 rows when every Lx is even; with the
    second-order advection scheme the cell kernel at 8 rows only."""
    lz = max(p.Lz for p in params)
    if params[0].advection:
        shapes = [(0, 8)]        # the second-order advection runs at 8-row tiles only
    else:
        shapes = [(0, ty) for ty in TILE_Y]
        if all(p.Lx % 2 == 0 for p in params):
            shapes.append((1, 16))
    return [(k, ty, zc) for k, ty in shapes for zc in Z_CHUNKS if zc <= lz]


def tune(params: Params | list[Params], steps: int = 12, cache: str | None = CACHE, device=None,
         rho: list | None = None, force: bool = False) -> dict:
    """Return ``{"kernel": .., "tile_y": .., "z_chunk": .., "ms_per_step": .., "trials": [...]}``
    for the batch ``params`` (a single instance or a list)."""
    import torch
    from . import lbfe
    plist = [params] if isinstance(params, Params) else list(params)
    dev = torch.device(device or "cuda")
    gpu = torch.cuda.get_device_name(dev)
    key = _key(plist, gpu)
    if cache and not force:
        hit = _load(cache).get(key)
        if hit:
            return hit
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        s = lbfe.Solver(plist, device=dev, stream=stream)
        for k, p in enumerate(plist):
            r = rho[k] if rho is not None else np.stack([np.full((p.Lz, p.Ly, p.Lx), p.rho_in),
                                                         np.full((p.Lz, p.Ly, p.Lx), p.rho_out)])
            s.init(k, r)
        trials = []
        for kern, ty, zc in candidates(plist):
            s.tune(ty, zc, kern)
            s.step(2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(steps)
            e1.record(stream)
            e1.synchronize()
            trials.append((kern, ty, zc, e0.elapsed_time(e1) / steps))
        s.close()
    best = min(trials, key=lambda t: t[3])
    out = {"kernel": best[0], "tile_y": best[1], "z_chunk": best[2], "ms_per_step": best[3],
           "trials": [list(t) for t in trials]}
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        data = _load(cache)
        data[key] = out
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1)
        os.replace(tmp, cache)
    return out
