"""The block order of the FP32 3-D tiled step (csrc/rlb_step_f32.cuh:
slab_order; csrc/rlb_step_f32.cu: f32_slab_rows), restated here and checked
on the CPU:

* for every grid of block rows and planes and every slab height, the remap
  from a block's linear index to its tile is a bijection onto the tiles
  (each tile is computed exactly once), including ragged last slabs;
* consecutive linear indices walk a slab plane by plane: within one slab
  the z-plane of a block never decreases as the linear index grows, and
  all tiles of slab s come before those of slab s + 1;
* the automatic slab height is the number of block rows whose f and h
  planes fill about 10 MB, at least 1 and at most the grid's block rows
  (16 at nx = 512).

The GPU tests (tests/test_gpu_slabs.py) show that every order gives the same
state bit for bit.
"""
import itertools

import pytest


def slab_order(L, nbx, nby, nbz, sb):
    """the tile (bx, by, bz) of the block with linear index L"""
    if sb == 0 or sb >= nby:
        bz, r = divmod(L, nbx * nby)
        by, bx = divmod(r, nbx)
        return bx, by, bz
    s = L // (nbx * sb * nbz)
    rows = min(sb, nby - s * sb)
    r = L - s * (nbx * sb * nbz)
    bz = r // (nbx * rows)
    q = r - bz * (nbx * rows)
    return q % nbx, s * sb + q // nbx, bz


def slab_rows(nx, ny, target_kb=10240, by=8):
    row_bytes = by * nx * 38 * 4
    nby = (ny + by - 1) // by
    s = int(target_kb * 1024 / row_bytes)
    return max(1, min(s, nby))


@pytest.mark.parametrize("nbx,nby,nbz", [(1, 1, 1), (8, 32, 4), (3, 5, 7), (2, 33, 3), (4, 12, 2)])
@pytest.mark.parametrize("sb", [0, 1, 2, 3, 4, 5, 16, 40])
def test_remap_is_a_bijection_in_slab_order(nbx, nby, nbz, sb):
    tiles = [slab_order(L, nbx, nby, nbz, sb) for L in range(nbx * nby * nbz)]
    assert sorted(tiles) == sorted(itertools.product(range(nbx), range(nby), range(nbz)))
    h = sb if 0 < sb < nby else nby
    prev_slab, prev_z = 0, 0
    for bx, by, bz in tiles:
        slab = by // h
        assert slab >= prev_slab
        if slab == prev_slab:
            assert bz >= prev_z
        else:
            prev_slab = slab
        prev_z = bz


def test_automatic_slab_height():
    assert slab_rows(512, 256) == 16       # the 512 x 256 x 256 cloud: two slabs
    assert slab_rows(1024, 96) == 8        # wider rows, thinner slabs (ragged: 8 + 4)
    assert slab_rows(128, 64) == 8         # narrow grid: one slab, the plain order
    assert slab_rows(1 << 20, 64) == 1     # at least one block row
    for nx in (64, 192, 512, 2048, 8192):
        s = slab_rows(nx, 1 << 14)
        assert s * 8 * nx * 38 * 4 <= 10240 * 1024 < (s + 1) * 8 * nx * 38 * 4 or s == 1
