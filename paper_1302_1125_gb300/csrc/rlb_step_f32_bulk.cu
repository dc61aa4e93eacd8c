// The FP32-storage step on 3-D grids with the stencil tiles staged by bulk
// copies (rlb_bulk.cuh), in a unit of its own so that it compiles in
// parallel with the other step kernels.  Eligible grids: viscous step, 19
// planes, extended lattice, nx a multiple of 64 and ny a multiple of 8 (every
// block a full 64 x 8 tile, so that all its threads take part in the
// barriers), x faces not periodic, and rlb_options.thread_mapping = 3 (an
// option); the launcher in rlb_step_f32.cu runs the per-thread staged kernel
// otherwise, and also when the tensor maps could not be made.
#include <cudaTypedefs.h>   // PFN_cuTensorMapEncodeTiled

#include "rlb_step_f32_launch.cuh"

namespace rlb {
namespace f32 {

constexpr int kBulkThreads = 256;   // 32 x 8
// dynamic shared memory: tiles, parked h coefficients, mbarriers, counters,
// the row and plane maps
constexpr size_t bulk_smem_bytes()
{
    return sizeof(float) * size_t(kBulkBufs) * kTileFloats + sizeof(f2) * size_t(kParkSlots) * kBulkThreads +
           sizeof(unsigned long long) * kBulkBufs + 2 * sizeof(int) * kBulkBufs + sizeof(int) * 16;
}

// maps: tensor maps of the f and h buffers the step reads
template <int LAT>
__global__ void __launch_bounds__(kBulkThreads, 2)
    step_f32_bulk_kernel(const StepParams p, const float *__restrict__ f, const float *__restrict__ h,
                         float *__restrict__ fo, float *__restrict__ ho, float *__restrict__ prev,
                         const __grid_constant__ TileMaps maps)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float *tiles = reinterpret_cast<float *>(smem);
    f2 *park = reinterpret_cast<f2 *>(smem + sizeof(float) * size_t(kBulkBufs) * kTileFloats);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(
        smem + sizeof(float) * size_t(kBulkBufs) * kTileFloats + sizeof(f2) * size_t(kParkSlots) * kBulkThreads);
    int *issued = reinterpret_cast<int *>(bars + kBulkBufs);
    int *done = issued + kBulkBufs;
    int *ymap = done + kBulkBufs, *zmap = ymap + 12;

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + 32 * ty;
    Bulk b;
    b.tile = tiles;
    b.full = bars;
    b.done = done;
    b.issued = issued;
    b.warp = ty;
    b.lane = tx;
    unsigned bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
    slab_order(p.slab_by, bx, by, bz);   // the per-thread staged kernel's block order
    b.x0t = 64 * int(bx);
    b.y0 = 8 * int(by);
    b.z = int(bz);
    b.cxlo = b.x0t == 0 ? 0 : b.x0t - 4;
    b.cxhi = b.x0t + 64 == p.nx ? p.nx : b.x0t + 68;
    b.ymap = ymap;
    b.zmap = zmap;
    b.maps = &maps;
    // tensor boxes read zeros outside the grid: tiles whose y halo crosses a
    // y face copy their centre rows row by row, through the boundary map
    b.rows = b.y0 < 2 || b.y0 + 10 > p.ny;
    b.failed = false;
    b.ctr = tiles + (ty + 2) * kRowC + 2 * tx + 4;
    b.zpl = tiles + kCentreFloats + ty * 64 + 2 * tx;
    if (tid == 0) {
        for (int k = 0; k < kBulkBufs; ++k) {
            mbar_init(&b.full[k], 1);
            issued[k] = 0;
            done[k] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid >= 32 && tid < 44) {
        ymap[tid - 32] = bulk_map(b.y0 - 2 + (tid - 32), p.ny, p.bc_lo[1], p.bc_hi[1]);
    } else if (tid >= 64 && tid < 68) {
        const int k = tid - 64;
        zmap[k] = bulk_map(b.z + (k < 2 ? k - 2 : k - 1), p.nz, p.bc_lo[2], p.bc_hi[2]);
    }
    __syncthreads();
    // the first kBulkBufs items, item j by warp j % 8, in flight while the
    // moment sums load
    for_pops(std::make_integer_sequence<int, kBulkBufs>{}, [&](auto jc) {
        constexpr int j = decltype(jc)::value;
        if (b.warp == j % 8) bulk_issue<19, j, LAT>(b, p, f, h);
    });

    const int x0 = b.x0t + 2 * tx, y = b.y0 + ty, z = b.z;
    Geo g;
    g.idx0 = x0 + p.nx * (y + p.ny * z);
    g.x0 = x0;
    g.has1 = true;
    g.idx1 = g.idx0 + 1;
    g.oa = 0;
    g.oc = 0;
    g.xfix = 0u;
    if (x0 == 0) g.xfix |= p.bc_lo[0] == BC_OUTFLOW ? XF_LO_CLAMP : XF_LO_GHOST;
    if (x0 + 2 >= p.nx) g.xfix |= p.bc_hi[0] == BC_OUTFLOW ? XF_HI_CLAMP : XF_HI_GHOST;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        g.yoff[k] = 0;   // the tile source takes neighbours by axis and distance
        g.zoff[k] = 0;
    }
    update_pair<3, false, true, LD_NC, kParkOn, false, 19, LAT, false, true>(
        p, g, p.f_eta_over_s, p.f_kbulk, f, h, fo, ho, prev, p.ps, park + tid, kBulkThreads, nullptr, 0, &b);

    // after a timeout: let the copies this block issued land before the
    // shared memory is released (bounded as well)
    if (__syncthreads_or(b.failed ? 1 : 0)) {   // every thread of the block takes part
        if (tid < kBulkBufs && issued[tid] > 0) mbar_wait(&b.full[tid], unsigned(issued[tid] - 1) & 1u);
        __syncthreads();
    }
}

}  // namespace f32

bool f32_bulk_eligible(const StepParams &p, int dim, int euler)
{
    return dim == 3 && !euler && p.sym == 0 && p.lat == 0 && p.mapping == 3 &&
           p.nx % 64 == 0 && p.ny % 8 == 0 && p.bc_lo[0] != BC_PERIODIC && p.bc_hi[0] != BC_PERIODIC;
}

cudaError_t make_tile_maps(const StepParams &p, const float *f, const float *h, TileMaps *out)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                               cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    // (x, y, z, population plane) of one distribution's 19 planes
    const cuuint64_t dims[4] = {cuuint64_t(p.nx), cuuint64_t(p.ny), cuuint64_t(p.nz), 19};
    const cuuint64_t strides[3] = {cuuint64_t(p.nx) * 4, cuuint64_t(p.nx) * p.ny * 4, cuuint64_t(p.ps) * 4};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const cuuint32_t boxc[4] = {f32::kRowC, 12, 1, 1};
    const cuuint32_t boxz[4] = {64, 8, 1, 1};
    auto make = [&](CUtensorMap *m, const float *base, const cuuint32_t *box) {
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    };
    if (make(&out->fc, f, boxc) != CUDA_SUCCESS || make(&out->fz, f, boxz) != CUDA_SUCCESS ||
        make(&out->hc, h, boxc) != CUDA_SUCCESS || make(&out->hz, h, boxz) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t launch_step_f32_bulk(const StepParams &p, const float *f, const float *h, float *fo, float *ho,
                                 float *prev, const TileMaps *maps, cudaStream_t s)
{
    const size_t smem = f32::bulk_smem_bytes();
    constexpr int kMaxDevices = 64;
    static std::atomic<bool> attr_set[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= kMaxDevices || !attr_set[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(f32::step_f32_bulk_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem));
        if (e != cudaSuccess) return e;
        if (dev < kMaxDevices) attr_set[dev].store(true, std::memory_order_release);
    }
    if (!maps) return cudaErrorInvalidValue;
    const dim3 block(32, 8, 1), grid(unsigned(p.nx / 64), unsigned(p.ny / 8), unsigned(p.nz));
    f32::step_f32_bulk_kernel<0><<<grid, block, smem, s>>>(p, f, h, fo, ho, prev, *maps);
    return cudaGetLastError();
}

}  // namespace rlb
