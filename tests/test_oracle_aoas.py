"""Pins of the CPU AoAoS <-> SoA conversion (paper Sec. II-B data layout,
Sec. III-C Eq. 4 gather prologue / scatter epilogue) against brute-force
pure-Python index loops written from the layout definition."""
import numpy as np
import pytest

from oracle import aoas
from paper_2608_19273_gb300 import synth


def code(k, x, y, z, v):
    """A unique value per (patch, voxel, quantity); halo voxels have coordinates outside [0, p)."""
    return float(k * 1_000_000 + (z + 10) * 10_000 + (y + 10) * 100 + (x + 10)) + v / 64.0


def make_case(dim, ps, nq, halo, pad=16):
    patches = np.zeros(len(ps), dtype=synth.PATCH_DTYPE)
    off = 0
    for k, p in enumerate(ps):
        patches[k]["p"] = p
        patches[k]["offset"] = off
        off += p ** dim + pad          # gaps between the patch blocks
    var_stride = off + 5
    blocks = []
    for k, p in enumerate(ps):
        ph = p + 2 * halo
        b = np.empty(aoas.block_len(p, dim, nq, halo))
        nz = ph if dim == 3 else 1
        for Z in range(nz):
            for Y in range(ph):
                for X in range(ph):
                    for v in range(nq):
                        vox = (Z * ph + Y) * ph + X
                        z = Z - halo if dim == 3 else 0
                        b[vox * nq + v] = code(k, X - halo, Y - halo, z, v)
        blocks.append(b)
    return patches, blocks, var_stride


@pytest.mark.parametrize("dim,ps,nq,halo", [(3, [2, 3, 2], 3, 0), (3, [3, 2], 2, 1), (3, [2], 1, 2),
                                           (2, [3, 4, 2], 4, 1), (2, [2], 5, 0)])
def test_gather_matches_index_definition(dim, ps, nq, halo):
    patches, blocks, vs = make_case(dim, ps, nq, halo)
    arena = np.full(nq * vs, -7.0)
    aoas.gather_aoas(patches, blocks, nq, halo, vs, dim, arena=arena)
    touched = np.zeros(nq * vs, dtype=bool)
    for k, p in enumerate(ps):
        off = int(patches[k]["offset"])
        for z in range(p if dim == 3 else 1):
            for y in range(p):
                for x in range(p):
                    for v in range(nq):
                        i = v * vs + off + (z * p + y) * p + x
                        assert arena[i] == code(k, x, y, z, v)
                        touched[i] = True
    assert np.all(arena[~touched] == -7.0)


@pytest.mark.parametrize("dim,ps,nq,halo", [(3, [2, 3], 3, 1), (2, [4, 2], 2, 2), (3, [2], 4, 0)])
def test_scatter_inverts_gather_and_keeps_halo(dim, ps, nq, halo):
    patches, blocks, vs = make_case(dim, ps, nq, halo)
    arena = aoas.gather_aoas(patches, blocks, nq, halo, vs, dim)
    out = [np.full_like(b, -3.0) for b in blocks]
    aoas.scatter_aoas(patches, arena, out, nq, halo, vs, dim)
    for k, p in enumerate(ps):
        ph = p + 2 * halo
        nz = ph if dim == 3 else 1
        for Z in range(nz):
            for Y in range(ph):
                for X in range(ph):
                    inside = all(halo <= c < halo + p for c in ((X, Y, Z) if dim == 3 else (X, Y)))
                    for v in range(nq):
                        j = ((Z * ph + Y) * ph + X) * nq + v
                        assert out[k][j] == (blocks[k][j] if inside else -3.0)
