// rlb_bulk.cuh -- block-level staging of the stencil tiles of the FP32 step by
// the copy engine (tensor-map bulk copies, cp.async.bulk.tensor), for 3-D
// grids.
//
// A block of 32 x 8 threads updates a tile of 64 x 8 cells in one z-plane
// (two x-adjacent cells per thread).  For each of its 38 items (f classes,
// then h classes) the block needs, from the population's plane:
//   the tile's own rows with the y neighbours the item streams or diffuses
//   over (rows y0 - 2 .. y0 + 9 at most), 72 values wide (x0 - 4 .. x0 + 67,
//   the x neighbours);
//   the tile's 8 rows in the z-neighbour planes it needs (z - 2, z - 1,
//   z + 1, z + 2 at most), 64 values wide.
// The centre rows arrive as one 72 x 12 tensor box, each z-neighbour plane as
// one 64 x 8 box, into one of kBulkBufs shared-memory buffers, completed on
// that buffer's "full" mbarrier (expect-tx with the item's byte count).  A
// tile whose y halo crosses a y face takes its centre rows as row copies
// (cp.async.bulk) from the rows the y boundary map picks (a 72 x 12 box
// would read zeros there; 72 x 1 boxes cannot land on rows that are not
// 128-byte aligned, as tensor copies into shared memory must).  The copies
// of item J + kBulkBufs go into item J's buffer once every warp is done with
// item J: each warp counts itself out on the buffer's counter (an atomic add
// after a release fence), and the warp that counts the last one issues
// them, a few lanes one copy each, so no warp waits for another to finish.
// Threads then read their stencil from the tile at fixed offsets: no
// per-thread address arithmetic and no per-thread copies.  The boundary maps
// of the block's rows and planes are computed once, into shared memory, so
// the issue of an item is a few instructions (the 38 items are unrolled:
// their code has to stay small enough for the instruction cache).
//
// At the grid's x ends the halo columns are not data (boxes read zeros
// there, row copies leave them alone), and the edge threads' clamp or ghost
// fix-ups replace them, so the x faces must not be periodic.
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
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// the box of tensor map `map` at element coordinates (x, y, z, plane) into
// shared dst (128-byte aligned), completing on bar with the box's full size
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
    const int *ymap;              // [12] (shared): grid row of centre row t (y0 - 2 + t through the y map)
    const int *zmap;              // [4] (shared): grid plane of z - 2, z - 1, z + 1, z + 2 through the z map
    int warp, lane;
    int x0t, y0, z;               // tile origin
    int cxlo, cxhi;               // x range of the centre row copies (the tile's x halo, inside the grid)
    const TileMaps *maps;         // tensor maps of f and h
    bool rows;                    // centre rows by row copies (a y-edge tile)
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
};

// issue the copies of item J into buffer J % kBulkBufs (called by a whole
// warp): lanes 0 .. nz - 1 the z-neighbour planes, lane 31 the centre box,
// or lanes 4 .. 4 + nc - 1 the centre rows of a y-edge tile
template <int NP, int J, int LAT>
__device__ __forceinline__ void bulk_issue(Bulk &b, const StepParams &p, const float *f, const float *h)
{
    using R = ItemRows<NP, J, LAT>;
    constexpr int buf = J % kBulkBufs;
    constexpr int nz = R::khi - R::klo;
    constexpr unsigned zbytes = unsigned(nz * kPlaneFloats * 4);
    const unsigned rowbytes = unsigned(b.cxhi - b.cxlo) * 4u;
    if (b.lane == 0) {
        mbar_expect_tx(&b.full[buf], b.rows ? unsigned(R::nc) * rowbytes + zbytes : unsigned(kCentreFloats * 4) + zbytes);
        b.issued[buf] += 1;
    }
    __syncwarp();
    float *dst0 = b.tile + buf * kTileFloats;
    if (b.lane < nz) {
        const int k = R::klo + b.lane;
        tma_g2s(dst0 + kCentreFloats + k * kPlaneFloats, R::IS_F ? &b.maps->fz : &b.maps->hz, b.x0t, b.y0, b.zmap[k],
                R::I, &b.full[buf]);
    }
    if (!b.rows) {
        if (b.lane == 31) tma_g2s(dst0, R::IS_F ? &b.maps->fc : &b.maps->hc, b.x0t - 4, b.y0 - 2, b.z, R::I, &b.full[buf]);
    } else if (b.lane >= 4 && b.lane < 4 + R::nc) {
        const int t = R::tlo + b.lane - 4;
        const float *q = (R::IS_F ? f : h) + R::I * p.ps;
        bulk_g2s(dst0 + t * kRowC + (b.cxlo - (b.x0t - 4)),
                 q + (long long)(b.z * p.ny + b.ymap[t]) * p.nx + b.cxlo, rowbytes, &b.full[buf]);
    }
}

}  // namespace f32
}  // namespace rlb
