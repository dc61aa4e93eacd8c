"""The copy plan of the bulk-staged FP32 step (csrc/rlb_bulk.cuh: ItemRows,
bulk_issue; csrc/rlb_step_f32_bulk.cu), restated here and checked on the CPU
on small eligible grids with every kind of face:

* every copy reads inside its population's plane (row copies) or starts its
  box at an x coordinate that is a multiple of 4 floats (16 bytes; the
  tensor boxes may start outside the grid, where they read zeros), with
  shared destinations 16-byte aligned and inside their buffer;
* the copies of one item do not overlap, and the bytes each item announces
  to its mbarrier (expect-tx) are the bytes its copies bring;
* every shared value a thread reads for an item was written by that item's
  copies, except the halo columns at the grid's x ends, which the edge
  threads' clamp or ghost fix-ups replace.

This is the check that ran before the kernel's first GPU run; the GPU tests
(tests/test_gpu_bulk.py) compare its results with the per-thread staged
kernel bit for bit.
"""
import itertools

import pytest

# the lattice vectors c_i of the extended lattice, in the library's order
DIRS = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (2, 2, 0), (2, -2, 0),
        (-2, 2, 0), (-2, -2, 0), (2, 0, 2), (2, 0, -2), (-2, 0, 2), (-2, 0, -2), (0, 2, 2), (0, 2, -2), (0, -2, 2),
        (0, -2, -2)]
NB, ROWC, CENTRE, PLANE = 6, 72, 12 * 72, 8 * 64
TILE = CENTRE + 4 * PLANE


def item_rows(J):
    is_f = J < 19
    I = J if is_f else J - 19
    lap = is_f and I != 0
    cx, cy, cz = DIRS[I]
    xneed = cx != 0 or lap
    tlo = 0 if cy > 0 else (1 if (cy < 0 or lap) else 2)
    thi = 12 if cy < 0 else (11 if (cy > 0 or lap) else 10)
    klo = 0 if cz > 0 else (1 if (cz < 0 or lap) else 4)
    khi = 4 if cz < 0 else (3 if (cz > 0 or lap) else 4)
    return I, lap, xneed, cy, cz, tlo, thi, klo, khi


def bmap(c, n, lo, hi):
    if 0 <= c < n:
        return c
    bc = lo if c < 0 else hi
    return c % n if bc == 0 else (0 if c < 0 else n - 1)


def plan(nx, ny, nz, lo, hi, tensor, bx, by, bz, J):
    """the copies of item J for the block (bx, by, bz): (dst, nfloats,
    source) with source ("row", first element offset in the plane) or
    ("box", x, y)"""
    I, lap, xneed, cy, cz, tlo, thi, klo, khi = item_rows(J)
    x0t, y0, z = 64 * bx, 8 * by, bz
    cxlo = 0 if x0t == 0 else x0t - 4
    cxhi = nx if x0t + 64 == nx else x0t + 68
    buf = J % NB
    rows = not tensor or y0 < 2 or y0 + 10 > ny
    out = []
    if tensor and not rows:
        out.append((buf * TILE, CENTRE, ("box", x0t - 4, y0 - 2)))
    else:
        xlo, xhi = (cxlo, cxhi) if xneed else (x0t, x0t + 64)
        for t in range(tlo, thi):
            y = bmap(y0 - 2 + t, ny, lo[1], hi[1])
            out.append((buf * TILE + t * ROWC + (xlo - (x0t - 4)), xhi - xlo, ("row", z * nx * ny + y * nx + xlo)))
    for k in range(klo, khi):
        d = k - 2 if k < 2 else k - 1
        zm = bmap(z + d, nz, lo[2], hi[2])
        if tensor:
            out.append((buf * TILE + CENTRE + k * PLANE, PLANE, ("box", x0t, y0)))
        else:
            for t in range(8):
                out.append((buf * TILE + CENTRE + k * PLANE + t * 64, 64,
                            ("row", zm * nx * ny + (y0 + t) * nx + x0t)))
        assert 0 <= zm < nz
    return out, rows


def expect_bytes(nx, ny, tensor, bx, by, J):
    I, lap, xneed, cy, cz, tlo, thi, klo, khi = item_rows(J)
    x0t, y0 = 64 * bx, 8 * by
    cxlo = 0 if x0t == 0 else x0t - 4
    cxhi = nx if x0t + 64 == nx else x0t + 68
    rowbytes = (cxhi - cxlo) * 4 if xneed else 256
    rows = not tensor or y0 < 2 or y0 + 10 > ny
    centre = (thi - tlo) * rowbytes if rows else CENTRE * 4
    return centre + (khi - klo) * PLANE * 4


GRIDS = [((64, 8, 2), (1, 1, 1), (1, 1, 1)), ((128, 16, 3), (2, 0, 1), (1, 0, 1)),
         ((64, 8, 5), (1, 0, 0), (2, 0, 0)), ((192, 32, 4), (2, 0, 0), (1, 0, 0))]


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("dims,lo,hi", GRIDS)
def test_bulk_copy_plan(dims, lo, hi, tensor):
    nx, ny, nz = dims
    N = nx * ny * nz
    for bx, by, bz in itertools.product(range(nx // 64), range(ny // 8), range(nz)):
        x0t = 64 * bx
        for J in range(38):
            I, lap, xneed, cy, cz, tlo, thi, klo, khi = item_rows(J)
            buf = J % NB
            copies, rows = plan(nx, ny, nz, lo, hi, tensor, bx, by, bz, J)
            written = {}
            total = 0
            for dst, n, src in copies:
                assert (dst * 4) % 16 == 0 and (n * 4) % 16 == 0
                assert buf * TILE <= dst and dst + n <= (buf + 1) * TILE
                if src[0] == "row":
                    assert 0 <= src[1] and src[1] + n <= N and (src[1] * 4) % 16 == 0
                else:
                    assert (src[1] * 4) % 16 == 0
                for e in range(dst, dst + n):
                    assert e not in written
                    written[e] = True
                total += 4 * n
            assert total == expect_bytes(nx, ny, tensor, bx, by, J)
            # the reads of every thread of the block
            for ty, tx in itertools.product(range(8), range(32)):
                x0 = x0t + 2 * tx
                ctr = buf * TILE + (ty + 2) * ROWC + 2 * tx + 4
                zpl = buf * TILE + CENTRE + ty * 64 + 2 * tx
                reads = [ctr, ctr + 1]
                if xneed:
                    if x0 != 0:
                        reads += [ctr - 2, ctr - 1]
                    if x0 + 2 < nx:
                        reads += [ctr + 2, ctr + 3]
                ydist = {1: (-2, -1, 1), -1: (-1, 1, 2)}.get(cy, (-1, 1) if lap else ())
                zdist = {1: (-2, -1, 1), -1: (-1, 1, 2)}.get(cz, (-1, 1) if lap else ())
                for d in ydist:
                    reads += [ctr + d * ROWC, ctr + d * ROWC + 1]
                for d in zdist:
                    k = d + 2 if d < 0 else d + 1
                    reads += [zpl + k * PLANE, zpl + k * PLANE + 1]
                for e in reads:
                    assert e in written, (dims, bx, by, bz, J, tx, ty, e)
