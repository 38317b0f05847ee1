"""AoAoS <-> SoA-arena conversion: the gather prologue and scatter epilogue of
the batched kernel (paper Sec. III-C, Eq. 4), on the CPU.

TEST INFRASTRUCTURE ONLY: the tests are the only users.  The CUDA library
never imports or calls anything here.

Layouts (paper Sec. II-B: each patch is one contiguous array of structs, the
K patches are not contiguous with each other; Sec. II Eq. 2: the cell kernel
sees p^ = p + 2h voxels per dimension, halo included):

* AoS block of patch k, halo width h, p^ = p + 2h: quantity v of voxel
  (x, y, z) -- halo-inclusive coordinates, z = 0 in 2D -- is element
  ((z * p^ + y) * p^ + x) * nq + v.
* SoA arena: quantity v of interior voxel (x, y, z) of patch k is element
  v * var_stride + offset_k + (z * p + y) * p + x.

gather copies the interior voxels of every block into the arena; scatter
copies them back.  Halo entries of the blocks are never read or written.
Both are plain permutations, written out as the index formula above with
numpy slicing (a reshape and an axis transpose per patch).
"""
from __future__ import annotations

import numpy as np


def block_len(p: int, dim: int, nq: int, halo: int) -> int:
    """Doubles in one AoS block: (p + 2h)^dim * nq."""
    return (p + 2 * halo) ** dim * nq


def _interior(block: np.ndarray, p: int, dim: int, nq: int, halo: int) -> np.ndarray:
    """View of the interior voxels of an AoS block, shape (p,)*dim + (nq,), axes (z, y, x, v)."""
    ph = p + 2 * halo
    b = block.reshape((ph,) * dim + (nq,))
    sl = (slice(halo, halo + p),) * dim
    return b[sl]


def gather_aoas(patches, blocks, nq: int, halo: int, var_stride: int, dim: int, arena=None) -> np.ndarray:
    """arena[v*vs + off_k + (z*p + y)*p + x] = block_k[((z+h)*p^ + y+h)*p^ + x+h)*nq + v].

    ``arena`` (nq * var_stride doubles) is updated in place when given, else
    created zero-filled; entries outside the patches' blocks stay untouched."""
    if arena is None:
        arena = np.zeros(nq * var_stride)
    a2 = arena.reshape(nq, var_stride)
    for k, pt in enumerate(patches):
        p, off = int(pt["p"]), int(pt["offset"])
        inner = _interior(np.asarray(blocks[k]), p, dim, nq, halo)   # (z, y, x, v) or (y, x, v)
        soa = np.moveaxis(inner, -1, 0).reshape(nq, p ** dim)          # (v, voxel in z-y-x order)
        a2[:, off:off + p ** dim] = soa
    return arena


def scatter_aoas(patches, arena: np.ndarray, blocks, nq: int, halo: int, var_stride: int, dim: int):
    """block_k[((z+h)*p^ + y+h)*p^ + x+h)*nq + v] = arena[v*vs + off_k + (z*p + y)*p + x], in place;
    halo entries of the blocks keep their values."""
    a2 = np.asarray(arena).reshape(nq, var_stride)
    for k, pt in enumerate(patches):
        p, off = int(pt["p"]), int(pt["offset"])
        inner = _interior(blocks[k], p, dim, nq, halo)
        soa = a2[:, off:off + p ** dim].reshape((nq,) + (p,) * dim)
        inner[...] = np.moveaxis(soa, 0, -1)
    return blocks
