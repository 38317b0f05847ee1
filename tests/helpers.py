"""Shared test helpers: arena <-> global-grid reshaping for single-level meshes."""
from __future__ import annotations

import numpy as np

from paper_2608_19273_gb300 import synth


def to_grid(mesh, row, li=0):
    """Arena row (var_stride,) -> global array [z][y][x] (2D: [y][x]) of level li."""
    lev = mesh.levels[li]
    p, dim = lev.p, mesh.dim
    nx, ny, nz = lev.n if dim == 3 else (lev.n[0], lev.n[1], 1)
    pz = p if dim == 3 else 1
    a, b = mesh.level_ranges[li]
    G = np.zeros((nz * pz, ny * p, nx * p))
    for k in range(a, b):
        r = k - a
        i, j, kk = r % nx, (r // nx) % ny, r // (nx * ny)
        off = int(mesh.patches[k]["offset"])
        blk = row[off:off + p * p * pz].reshape(pz, p, p)
        G[kk * pz:(kk + 1) * pz, j * p:(j + 1) * p, i * p:(i + 1) * p] = blk
    return G if dim == 3 else G[0]


def from_grid(mesh, G, row, li=0):
    """Inverse of to_grid: write the global array of level li into an arena row."""
    lev = mesh.levels[li]
    p, dim = lev.p, mesh.dim
    nx, ny, nz = lev.n if dim == 3 else (lev.n[0], lev.n[1], 1)
    pz = p if dim == 3 else 1
    G3 = G if dim == 3 else G[None]
    a, b = mesh.level_ranges[li]
    for k in range(a, b):
        r = k - a
        i, j, kk = r % nx, (r // nx) % ny, r // (nx * ny)
        off = int(mesh.patches[k]["offset"])
        row[off:off + p * p * pz] = G3[kk * pz:(kk + 1) * pz, j * p:(j + 1) * p, i * p:(i + 1) * p].ravel()
    return row


def arena(mesh, nvar):
    return np.zeros((nvar, mesh.var_stride))


def single_level(n, p, dx, dim=3):
    return synth.make_mesh([synth.Level(n, p, dx, 0)], dim=dim)


def voxel_mask(mesh):
    """Boolean (var_stride,) marking arena entries that belong to a voxel (not padding)."""
    m = np.zeros(mesh.var_stride, dtype=bool)
    for pt in mesh.patches:
        n = int(pt["p"]) ** mesh.dim
        m[int(pt["offset"]):int(pt["offset"]) + n] = True
    return m
