"""Seeded synthetic inputs: initial component densities of a droplet in a box.

This module holds no arithmetic of the method itself; it only draws the
initial density fields that both the CUDA path and the CPU oracle start from,
so that neither needs the other's random numbers.

Recipe (one NumPy PCG64 stream, ``numpy.random.default_rng(seed)``, drawn in
this order):
  1. the droplet centre offset, 3 draws U(-1/2, 1/2) added to the box centre
     ((Lx-1)/2, (Ly-1)/2, (Lz-1)/2) (cell centres sit at integer coordinates,
     the walls at z = -1/2 and z = Lz - 1/2);
  2. the noise, ``2*Lz*Ly*Lx`` draws U(-a, a) in ``[component][z][y][x]``
     order.
A cell is inside the droplet when its centre lies within distance R of the
droplet centre (ties inside).  Component A (droplet) has density ``rho_in``
inside and ``rho_out`` outside; component B (matrix) the mirror image.
"""
from __future__ import annotations

import numpy as np


def droplet_densities(Lx: int, Ly: int, Lz: int, R: float, rho_in: float = 1.0,
                      rho_out: float = 0.04, noise: float = 1e-4, seed: int = 1,
                      center_offset: bool = True) -> np.ndarray:
    """Return ``rho[2][Lz][Ly][Lx]`` (float64) for one spherical droplet."""
    rng = np.random.default_rng(seed)
    off = rng.uniform(-0.5, 0.5, size=3) if center_offset else np.zeros(3)
    cx, cy, cz = (Lx - 1) / 2 + off[0], (Ly - 1) / 2 + off[1], (Lz - 1) / 2 + off[2]
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    inside = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= R * R
    rho = np.empty((2, Lz, Ly, Lx))
    rho[0] = np.where(inside, rho_in, rho_out)
    rho[1] = np.where(inside, rho_out, rho_in)
    if noise > 0:
        rho += rng.uniform(-noise, noise, size=rho.shape)
    return rho


def cylinder_densities(Lx: int, Ly: int, Lz: int, R: float, rho_in: float = 1.0,
                       rho_out: float = 0.04) -> np.ndarray:
    """Droplet that is a cylinder along y (for the two-dimensional Laplace test)."""
    cx, cz = (Lx - 1) / 2, (Lz - 1) / 2
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    inside = (x - cx) ** 2 + (z - cz) ** 2 <= R * R
    rho = np.empty((2, Lz, Ly, Lx))
    rho[0] = np.where(inside, rho_in, rho_out)
    rho[1] = np.where(inside, rho_out, rho_in)
    return rho


def slab_densities(Lx: int, Ly: int, Lz: int, width: int, rho_in: float = 1.0,
                   rho_out: float = 0.04) -> np.ndarray:
    """Flat layer of component A, ``width`` planes thick, centred in x."""
    x0 = (Lx - width) // 2
    rho = np.empty((2, Lz, Ly, Lx))
    rho[0] = rho_out
    rho[1] = rho_in
    rho[0, :, :, x0:x0 + width] = rho_in
    rho[1, :, :, x0:x0 + width] = rho_out
    return rho


def random_state(Lx: int, Ly: int, Lz: int, seed: int, amp: float = 0.05):
    """Arbitrary smooth-ish populations and conformation tensor for unit tests.

    Returns ``(rho, vel, C)``: positive densities ``[2][Lz][Ly][Lx]``, a small
    velocity ``[3][Lz][Ly][Lx]`` and a symmetric positive-definite ``C``
    ``[6][Lz][Ly][Lx]`` (xx, yy, zz, xy, xz, yz).
    """
    rng = np.random.default_rng(seed)
    shp = (Lz, Ly, Lx)
    rho = np.empty((2,) + shp)
    rho[0] = 0.5 + rng.uniform(0, 0.5, shp)
    rho[1] = 0.5 - rho[0] + 0.55 + rng.uniform(0, 0.05, shp)
    vel = rng.uniform(-amp, amp, (3,) + shp)
    Lm = rng.uniform(-0.3, 0.3, (3, 3) + shp)
    Lm[0, 0] += 1.0; Lm[1, 1] += 1.0; Lm[2, 2] += 1.0
    Cfull = np.einsum("ik...,jk...->ij...", Lm, Lm)
    C = np.stack([Cfull[0, 0], Cfull[1, 1], Cfull[2, 2], Cfull[0, 1], Cfull[0, 2], Cfull[1, 2]])
    return rho, vel, C
