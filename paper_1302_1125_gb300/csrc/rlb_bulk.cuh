// rlb_bulk.cuh -- block-level staging of the stencil tiles of the FP32 step by
// bulk copies (the GB300 copy engine, cp.async.bulk), for 3-D grids.
//
// A block of 32 x 8 threads updates a tile of 64 x 8 cells in one z-plane
// (two x-adjacent cells per thread).  For each of its 38 items (f classes,
// then h classes) the block needs, from the population's plane:
//   the tile's own rows with the y neighbours the item streams or diffuses
//   over (rows y0 - 2 .. y0 + 9 at most), 72 values wide (x0 - 4 .. x0 + 67,
//   the x neighbours) or 64 when the item does not move along x and has no
//   Laplacian there;
//   the tile's 8 rows in the z-neighbour planes it needs (z - 2, z - 1,
//   z + 1, z + 2 at most), 64 values wide.
// Each such row segment is one bulk copy (288 or 256 bytes, 16-byte aligned)
// from global memory into one of kBulkBufs shared-memory buffers, completed
// on that buffer's "full" mbarrier (expect-tx with the item's byte count).
// The copies of item J + kBulkBufs go into item J's buffer once every warp
// is done with item J: each warp counts itself out on the buffer's counter
// (an atomic add after a release fence), and the warp that counts the last
// one issues them, its lanes one copy each, so no warp waits for another to
// finish.  Threads then read their stencil from the tile at fixed offsets:
// no per-thread address arithmetic and no per-thread copies.
// With tensor maps (the default) the centre rows are one 72 x 12 box and each
// z-neighbour plane one 64 x 8 box; tiles whose y halo crosses a y face, or
// grids without maps, copy the centre rows row by row.
//
// Source rows are chosen through the y and z boundary maps (periodic wrap or
// zero-gradient clamp), so the tile holds the mapped neighbours.  The x
// faces must not be periodic: at the grid's x ends the halo columns are not
// copied, and the edge threads' clamp or ghost fix-ups replace them.
//
// Every wait is bounded (about a second of clock cycles): on a timeout the
// thread sets ST_TIMEOUT in the status word, stops waiting and issuing, and
// the block drains the copies it issued (again bounded) before it exits.
#pragma once

#include <cuda_runtime.h>

#include "rlb_classes.cuh"
#include "rlb_device.cuh"
#include "rlb_internal.h"
#include "rlb_pair.cuh"

namespace rlb {
namespace f32 {

#ifndef RLB_BULK_BUFS
#define RLB_BULK_BUFS 6
#endif
constexpr int kBulkBufs = RLB_BULK_BUFS;     // items in flight
constexpr int kRowC = 72;                    // floats per centre row (x0 - 4 .. x0 + 67)
constexpr int kCentreFloats = 12 * kRowC;    // rows y0 - 2 .. y0 + 9
constexpr int kPlaneFloats = 8 * 64;         // one z-neighbour plane of the tile
constexpr int kTileFloats = kCentreFloats + 4 * kPlaneFloats;
constexpr long long kWaitCycles = 1LL << 31; // bound of every wait (~1 s)

__device__ __forceinline__ unsigned smem_addr(const void *p) { return unsigned(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}
// wait for the phase of the given parity to complete; false after kWaitCycles
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}
// bytes (a multiple of 16) from global src to shared dst (both 16-byte
// aligned), completing as transaction bytes on bar
__device__ __forceinline__ void bulk_g2s(float *dst, const float *src, unsigned bytes, unsigned long long *bar)
{
#ifdef RLB_BULK_DST_CLUSTER
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
#else
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
#endif
}
// the box of tensor map `map` at element coordinates (x, y, z, plane) into
// shared dst (16-byte aligned), completing on bar with the box's full size
// (elements outside the tensor arrive as zeros)
__device__ __forceinline__ void tma_g2s(float *dst, const CUtensorMap *map, int x, int y, int z, int plane,
                                        unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(plane), "r"(smem_addr(bar))
        : "memory");
}

// the block's staging state, in registers of each thread
struct Bulk {
    float *tile;                  // buffer 0 of the tiles (shared)
    const float *ctr;             // this thread's pair in the centre rows of buffer 0: row ty + 2, column 2 tx + 4
    const float *zpl;             // this thread's pair in z-plane 0 of buffer 0: row ty, column 2 tx
    unsigned long long *full;     // [kBulkBufs] (shared)
    int *done;                    // [kBulkBufs] (shared): warps that finished with each buffer, cumulative
    int *issued;                  // [kBulkBufs] (shared): phases issued per buffer
    int warp, lane;
    int x0t, y0, z;               // tile origin
    int cxlo, cxhi;               // x range copied into centre rows that need the x neighbours
    const TileMaps *maps;         // tensor maps of f and h (null: row-by-row copies)
    bool rows;                    // centre rows copied row by row (no maps, or a y-edge tile)
    bool failed;
};

// stencil values from the tile of one buffer (the Src interface of streamed2)
struct TileSrc {
    const float *ctr, *zpl;
    __device__ __forceinline__ f2 get(int slot, int) const
    {
        const float2 v = *reinterpret_cast<const float2 *>(ctr + 2 * (slot - 1));
        return f2{v.x, v.y};
    }
    template <int A, int D>
    __device__ __forceinline__ f2 nb(int, int) const
    {
        static_assert(A == 1 || A == 2, "x neighbours come through get");
        static_assert(D == -2 || D == -1 || D == 1 || D == 2, "distance 1 or 2");
        const float *q;
        if constexpr (A == 1) q = ctr + D * kRowC;
        else q = zpl + (D < 0 ? D + 2 : D + 1) * kPlaneFloats;
        const float2 v = *reinterpret_cast<const float2 *>(q);
        return f2{v.x, v.y};
    }
};

__device__ __forceinline__ int bulk_map(int c, int n, int lo, int hi)
{
    if (c >= 0 && c < n) return c;
    const int bc = c < 0 ? lo : hi;
    if (bc == BC_PERIODIC) {
        const int m = c % n;
        return m < 0 ? m + n : m;
    }
    return c < 0 ? 0 : n - 1;   // zero gradient (inlets are x faces only)
}

// rows of item J: centre tile rows [tlo, thi) (row t is y0 - 2 + t) and
// z-neighbour planes [klo, khi) of (z - 2, z - 1, z + 1, z + 2)
template <int NP, int J, int LAT>
struct ItemRows {
    static constexpr bool IS_F = J < NP;
    static constexpr int I = rep<NP>(IS_F ? J : J - NP);
    static constexpr bool lap = IS_F && I != 0;
    static constexpr bool xneed = cdir<I, 0, LAT>() != 0 || lap;
    static constexpr int cy = cdir<I, 1, LAT>(), cz = cdir<I, 2, LAT>();
    static constexpr int tlo = cy > 0 ? 0 : ((cy < 0 || lap) ? 1 : 2);
    static constexpr int thi = cy < 0 ? 12 : ((cy > 0 || lap) ? 11 : 10);
    static constexpr int klo = cz > 0 ? 0 : ((cz < 0 || lap) ? 1 : 4);
    static constexpr int khi = cz < 0 ? 4 : ((cz > 0 || lap) ? 3 : 4);
    static constexpr int nc = thi - tlo;
    static constexpr int nrows = nc + 8 * (khi - klo);
};

// issue the copies of item J into buffer J % kBulkBufs (called by a whole warp)
template <int NP, int J, int LAT>
__device__ __forceinline__ void bulk_issue(Bulk &b, const StepParams &p, const float *f, const float *h, long long ps)
{
    using R = ItemRows<NP, J, LAT>;
    constexpr int buf = J % kBulkBufs;
    if (b.maps) {
        // tensor boxes: the 72 x 12 centre tile (unless the tile's y halo
        // needs the boundary map: row copies below) and one 64 x 8 box per
        // z-neighbour plane
        constexpr int nz = R::khi - R::klo;
        const unsigned cbytes = b.rows ? unsigned(R::nc) * unsigned((R::xneed ? b.cxhi - b.cxlo : 64) * 4)
                                       : unsigned(kCentreFloats * 4);
        if (b.lane == 0) {
            mbar_expect_tx(&b.full[buf], cbytes + unsigned(nz) * unsigned(kPlaneFloats * 4));
            b.issued[buf] += 1;
        }
        __syncwarp();
        const CUtensorMap *mc = R::IS_F ? &b.maps->fc : &b.maps->hc;
        const CUtensorMap *mz = R::IS_F ? &b.maps->fz : &b.maps->hz;
        float *dst0 = b.tile + buf * kTileFloats;
        if (b.lane < nz) {
            const int k = R::klo + b.lane;
            const int d = k < 2 ? k - 2 : k - 1;
            const int zm = bulk_map(b.z + d, p.nz, p.bc_lo[2], p.bc_hi[2]);
            tma_g2s(dst0 + kCentreFloats + k * kPlaneFloats, mz, b.x0t, b.y0, zm, R::I, &b.full[buf]);
        }
        if (!b.rows) {
            if (b.lane == 31) tma_g2s(dst0, mc, b.x0t - 4, b.y0 - 2, b.z, R::I, &b.full[buf]);
        } else if (b.lane < R::nc) {
            const int xlo = R::xneed ? b.cxlo : b.x0t;
            const int t = R::tlo + b.lane;
            const int y = bulk_map(b.y0 - 2 + t, p.ny, p.bc_lo[1], p.bc_hi[1]);
            const float *q = (R::IS_F ? f : h) + R::I * ps;
            bulk_g2s(dst0 + t * kRowC + (xlo - (b.x0t - 4)), q + b.z * (long long)p.nx * p.ny + (long long)y * p.nx + xlo,
                     cbytes / unsigned(R::nc), &b.full[buf]);
        }
        return;
    }
    const int xlo = R::xneed ? b.cxlo : b.x0t;
    const int xhi = R::xneed ? b.cxhi : b.x0t + 64;
    const unsigned cbytes = unsigned(xhi - xlo) * 4u;
    if (b.lane == 0) {
        mbar_expect_tx(&b.full[buf], unsigned(R::nc) * cbytes + unsigned(R::nrows - R::nc) * 256u);
        b.issued[buf] += 1;
    }
    __syncwarp();
    const float *q = (R::IS_F ? f : h) + R::I * ps;
    float *dst0 = b.tile + buf * kTileFloats;
    const long long plane = (long long)p.nx * p.ny;
    for (int r = b.lane; r < R::nrows; r += 32) {
        if (r < R::nc) {
            const int t = R::tlo + r;
            const int y = bulk_map(b.y0 - 2 + t, p.ny, p.bc_lo[1], p.bc_hi[1]);
            bulk_g2s(dst0 + t * kRowC + (xlo - (b.x0t - 4)), q + b.z * plane + (long long)y * p.nx + xlo, cbytes,
                     &b.full[buf]);
        } else {
            const int rr = r - R::nc;
            const int k = R::klo + rr / 8, t = rr % 8;
            const int d = k < 2 ? k - 2 : k - 1;
            const int zm = bulk_map(b.z + d, p.nz, p.bc_lo[2], p.bc_hi[2]);
            bulk_g2s(dst0 + kCentreFloats + k * kPlaneFloats + t * 64,
                     q + zm * plane + (long long)(b.y0 + t) * p.nx + b.x0t, 256u, &b.full[buf]);
        }
    }
}

}  // namespace f32
}  // namespace rlb
