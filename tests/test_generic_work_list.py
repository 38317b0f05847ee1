"""Host logic of the generic FV stage's work list (dh_generic_work_list, no GPU): every voxel of
every patch belongs to exactly one work item, every item keeps within the kernel's shared-memory
limits, 2x2x2 blocks of 3^3 patches are formed only from patches that are each other's face
neighbours both ways, and the list runs largest item first.

Limits of one item (ng groups of bx x by x bz voxels): at most 256 voxels, 512 box cells with the
one-voxel face halo, 320 line cells and 256 faces of one direction."""
import numpy as np
import pytest

from helpers import single_level
from paper_2608_19273_gb300 import dh, synth


def _limits_ok(bx, by, bz, ng, dim):
    ez = 2 if dim == 3 else 0
    if ng * bx * by * bz > 256 or ng * (bx + 2) * (by + 2) * (bz + ez) > 512:
        return False
    for d in range(dim):
        lines = (bx + 2 * (d == 0)) * (by + 2 * (d == 1)) * (bz + 2 * (d == 2))
        faces = (bx + (d == 0)) * (by + (d == 1)) * (bz + (d == 2))
        if ng * lines > 320 or ng * faces > 256:
            return False
    return True


def _check(mesh, dim):
    P = mesh.patches
    items = dh.dh_generic_work_list(dim, P)
    assert len(items) > 0
    cost = items[:, 14] * items[:, 11] * items[:, 12] * items[:, 13]
    assert np.all(np.diff(cost) <= 0), "largest work first"
    whole = np.zeros(len(P), dtype=np.int64)       # times a patch is covered whole
    boxes = {}                                       # patch -> list of boxes
    for it in items:
        patch, (x0, y0, z0, bx, by, bz, ng, mp) = it[:8], it[8:]
        if mp:
            assert mp == 3 and (bx, by, bz, ng) == (6, 6, 6, 1) and dim == 3
            m = [int(k) for k in patch]
            assert len(set(m)) == 8
            for x in range(8):
                assert P[m[x]]["p"] == 3
                for ax in range(3):
                    hi = (x >> ax) & 1
                    # the member on the low side has its partner as +ax neighbour, and vice versa
                    assert P[m[x]]["nbr"][2 * ax + (0 if hi else 1)] == m[x ^ (1 << ax)]
                whole[m[x]] += 1
            continue
        assert _limits_ok(bx, by, bz, ng, dim), (bx, by, bz, ng)
        used = [int(k) for k in patch[:ng]]
        assert all(k >= 0 for k in used) and np.all(patch[ng:] == -1)
        if ng > 1 or (x0, y0, z0) == (0, 0, 0) and P[used[0]]["p"] == bx == by and (dim == 2 or bz == bx):
            # whole patches of one size
            for k in used:
                assert P[k]["p"] == bx == by and (bz == (bx if dim == 3 else 1))
                whole[k] += 1
        else:
            boxes.setdefault(used[0], []).append((x0, y0, z0, bx, by, bz))
    for k in range(len(P)):
        p = int(P[k]["p"])
        if k not in boxes:
            assert whole[k] == 1, f"patch {k} covered {whole[k]} times"
            continue
        assert whole[k] == 0
        bl = boxes[k]
        pz = p if dim == 3 else 1
        # the boxes are the product of one partition of [0, p) per axis
        parts = []
        for a, (o, e, n) in enumerate([(0, 3, p), (1, 4, p), (2, 5, pz)]):
            segs = sorted({(b[o], b[e]) for b in bl})
            pos = 0
            for s0, sl in segs:
                assert s0 == pos and sl > 0
                pos += sl
            assert pos == n
            parts.append(len(segs))
        assert len(bl) == len({b[:3] for b in bl}) == parts[0] * parts[1] * parts[2]
    return items


def test_blocks_of_3cubed_patches():
    mesh = single_level((4, 4, 4), 3, 1.0 / 48)
    items = _check(mesh, 3)
    assert len(items) == 8 and np.all(items[:, 15] == 3)


def test_blocks_and_leftovers():
    # 3 x 3 x 3 patches: one block; the other 19 patches go whole, four to an item
    items = _check(single_level((3, 3, 3), 3, 1.0 / 48), 3)
    assert np.sum(items[:, 15] == 3) == 1
    left = items[items[:, 15] == 0]
    assert sorted(left[:, 14].tolist(), reverse=True) == [4, 4, 4, 4, 3]
    # a patch that is its own z neighbour forms no block
    items = _check(single_level((2, 2, 1), 3, 1.0 / 48), 3)
    assert np.all(items[:, 15] == 0) and items[:, 14].sum() == 4


def test_mixed_sizes():
    mesh = synth.make_mesh([synth.Level((4, 4, 4), 3, 1.0 / 48, 0), synth.Level((2, 1, 1), 16, 1.0 / 32, 1),
                            synth.Level((2, 2, 2), 6, 1.0 / 40, 2)], dim=3)
    _check(mesh, 3)


@pytest.mark.parametrize("dim", [2, 3])
def test_patch_sizes(dim):
    """Every size up to 64 and a spread of larger ones, up to the largest (256)."""
    sizes = list(range(2, 65)) + list(range(67, 256, 9)) + [255, 256]
    for p in sizes:
        _check(single_level((1, 1, 1) if dim == 3 else (1, 1), p, 1.0 / p, dim=dim), dim)


def test_bad_tables_refused():
    mesh = single_level((2, 2, 2), 6, 1.0 / 12)
    bad = mesh.patches.copy()
    bad["nbr"][0, 1] = len(bad)
    with pytest.raises(dh.DhError) as e:
        dh.dh_generic_work_list(3, bad)
    assert e.value.status == dh.DH_EINVAL
    bad = mesh.patches.copy()
    bad["p"][0] = 257
    with pytest.raises(dh.DhError):
        dh.dh_generic_work_list(3, bad)
