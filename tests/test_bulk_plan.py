"""The copy plan of the bulk-staged FP32 step (csrc/rlb_bulk.cuh: ItemRows,
bulk_issue; csrc/rlb_step_f32_bulk.cu), restated here and checked on the CPU
on small eligible grids with every kind of face:

* every tensor box starts at an x coordinate that is a multiple of 4 floats
  (16 bytes; boxes may start outside the grid in x, where they read zeros)
  and at y and z coordinates inside the grid, and lands on a 128-byte
  aligned shared address; every row copy (the centre rows of tiles whose y
  halo crosses a y face) reads inside its population's plane, 16-byte
  aligned at both ends; all destinations are inside their buffer; the lanes
  that issue are distinct;
* the copies of one item do not overlap, and the bytes each item announces
  to its mbarrier (expect-tx) are the bytes its copies bring;
* every shared value a thread reads for an item holds the grid value the
  thread's stencil needs there: its neighbour along the item's axes, taken
  through the y and z boundary maps (periodic wrap or zero-gradient clamp).
  The halo columns at the grid's x ends are the exception: there the tile
  holds zeros, and the edge threads' clamp or ghost fix-ups replace them.

This is the check that runs before the kernel's GPU runs; the GPU tests
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
PERIODIC = 0


def sign(v):
    return (v > 0) - (v < 0)


def item_rows(J):
    is_f = J < 19
    I = J if is_f else J - 19
    lap = is_f and I != 0
    sx, sy, sz = (sign(c) for c in DIRS[I])
    xneed = sx != 0 or lap
    tlo = 0 if sy > 0 else (1 if (sy < 0 or lap) else 2)
    thi = 12 if sy < 0 else (11 if (sy > 0 or lap) else 10)
    klo = 0 if sz > 0 else (1 if (sz < 0 or lap) else 4)
    khi = 4 if sz < 0 else (3 if (sz > 0 or lap) else 4)
    return I, lap, xneed, sy, sz, tlo, thi, klo, khi


def bmap(c, n, lo, hi):
    """the grid index a y or z coordinate outside the grid maps to"""
    if 0 <= c < n:
        return c
    bc = lo if c < 0 else hi
    return c % n if bc == PERIODIC else (0 if c < 0 else n - 1)


def stencil_distances(s, lap):
    """neighbour distances a thread reads along one axis: the upwind
    flux-limited stencil of a population moving with sign s, the Laplacian's
    +-1"""
    d = set({1: (-2, -1, 1), -1: (-1, 1, 2)}.get(s, ()))
    if lap:
        d |= {-1, 1}
    return sorted(d)


def plan(nx, ny, nz, lo, hi, bx, by, bz, J):
    """the copies of item J for the block (bx, by, bz), as
    (lane, kind, shared destination, width, height, origin (x, y, z)):
    kind "box" a tensor box, "row" a row copy of `width` floats"""
    I, lap, xneed, sy, sz, tlo, thi, klo, khi = item_rows(J)
    x0t, y0, z = 64 * bx, 8 * by, bz
    ymap = [bmap(y0 - 2 + t, ny, lo[1], hi[1]) for t in range(12)]
    zmap = [bmap(z + (k - 2 if k < 2 else k - 1), nz, lo[2], hi[2]) for k in range(4)]
    buf = J % NB
    rows = y0 < 2 or y0 + 10 > ny
    out = []
    cxlo = 0 if x0t == 0 else x0t - 4
    cxhi = nx if x0t + 64 == nx else x0t + 68
    for lane in range(khi - klo):
        k = klo + lane
        out.append((lane, "box", buf * TILE + CENTRE + k * PLANE, 64, 8, (x0t, y0, zmap[k])))
    if not rows:
        out.append((31, "box", buf * TILE, ROWC, 12, (x0t - 4, y0 - 2, z)))
    else:
        for t in range(tlo, thi):
            out.append((4 + t - tlo, "row", buf * TILE + t * ROWC + (cxlo - (x0t - 4)), cxhi - cxlo, 1,
                        (cxlo, ymap[t], z)))
    expect = (thi - tlo) * (cxhi - cxlo) * 4 if rows else CENTRE * 4
    expect += (khi - klo) * PLANE * 4
    return out, expect


GRIDS = [((64, 8, 2), (1, 1, 1), (1, 1, 1)), ((128, 16, 3), (2, 0, 1), (1, 0, 1)),
         ((64, 8, 5), (1, 0, 0), (2, 0, 0)), ((192, 32, 4), (2, 0, 0), (1, 0, 0)),
         ((128, 24, 3), (1, 1, 0), (1, 1, 0))]


@pytest.mark.parametrize("dims,lo,hi", GRIDS)
def test_bulk_copy_plan(dims, lo, hi):
    nx, ny, nz = dims
    for bx, by, bz in itertools.product(range(nx // 64), range(ny // 8), range(nz)):
        x0t, y0 = 64 * bx, 8 * by
        for J in range(38):
            I, lap, xneed, sy, sz, tlo, thi, klo, khi = item_rows(J)
            buf = J % NB
            copies, expect = plan(nx, ny, nz, lo, hi, bx, by, bz, J)
            lanes = [c[0] for c in copies]
            assert len(set(lanes)) == len(lanes) and all(0 <= ln < 32 for ln in lanes)
            held = {}   # shared element -> the grid value it holds: (x, y, z), or None (zero fill)
            total = 0
            for _, kind, dst, w, hgt, (ox, oy, oz) in copies:
                assert (dst * 4) % (128 if kind == "box" else 16) == 0 and (w * 4) % 16 == 0
                assert (TILE * 4) % 128 == 0   # every buffer starts 128-byte aligned
                assert buf * TILE <= dst and dst + w * hgt <= (buf + 1) * TILE
                assert (ox * 4) % 16 == 0, "x start not 16-byte aligned"
                assert 0 <= oy and oy + hgt <= ny and 0 <= oz < nz
                if kind == "row":
                    assert 0 <= ox and ox + w <= nx
                for j, i in itertools.product(range(hgt), range(w)):
                    e = dst + j * w + i
                    assert e not in held
                    held[e] = (ox + i, oy + j, oz) if 0 <= ox + i < nx else None
                total += 4 * w * hgt
            assert total == expect
            # the reads of every thread of the block, with the value each needs
            z = bz
            for ty, tx in itertools.product(range(8), range(32)):
                x0 = x0t + 2 * tx
                y = y0 + ty
                ctr = buf * TILE + (ty + 2) * ROWC + 2 * tx + 4
                zpl = buf * TILE + CENTRE + ty * 64 + 2 * tx
                reads = []   # (shared element, grid value needed; None: replaced by an edge fix-up)
                for e in range(2):
                    reads.append((ctr + e, (x0 + e, y, z)))
                if xneed:
                    for e in range(-2, 4):
                        if e in (0, 1):
                            continue
                        xs = x0 + e
                        reads.append((ctr + e, (xs, y, z) if 0 <= xs < nx else None))
                for d in stencil_distances(sy, lap):
                    for e in range(2):
                        reads.append((ctr + d * ROWC + e, (x0 + e, bmap(y + d, ny, lo[1], hi[1]), z)))
                for d in stencil_distances(sz, lap):
                    k = d + 2 if d < 0 else d + 1
                    for e in range(2):
                        reads.append((zpl + k * PLANE + e, (x0 + e, y, bmap(z + d, nz, lo[2], hi[2]))))
                for e, need in reads:
                    if need is None:
                        assert x0 == 0 or x0 + 2 >= nx   # only the edge threads' replaced halo columns
                        continue
                    assert e in held, (dims, bx, by, bz, J, tx, ty, e)
                    assert held[e] == need, (dims, bx, by, bz, J, tx, ty, held[e], need)
