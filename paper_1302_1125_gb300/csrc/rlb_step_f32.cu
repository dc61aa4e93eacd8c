// FP32-storage form of the fused step (see rlb_step_f32.cuh): populations
// stored, streamed and relaxed in float, two cells per thread, double-float
// moment sums, no FP64 instructions.
#include <atomic>

#include "rlb_step_f32.cuh"

namespace rlb {

template <int DIM, bool EULER, bool VEC2, int LAT>
static cudaError_t launch_f32(const StepParams &p, const float *f, const float *h, float *fo, float *ho,
                             float *prev, cudaStream_t s)
{
    const int npairs = (p.nx + 1) / 2;
    dim3 block, grid;
    if (DIM == 1) {
        block = dim3(128, 1, 1);
        grid = dim3((npairs + 127) / 128, 1, 1);
    } else {
        // tiles of 32 x 8 threads (64 x 8 cells), two blocks per SM at <= 128
        // registers: the best of a sweep over block shapes and register caps on
        // GB300 when nx fills them; otherwise the same 256 threads take 256
        // consecutive pairs of the x-fastest order (the kernel reads the
        // mapping from the block shape)
        const long long tiles_x = (npairs + 31) / 32, tiles_y = (p.ny + RLB_F32_BY - 1) / RLB_F32_BY;
        const long long pairs = (long long)npairs * p.ny * p.nz;
        const double fill = double(npairs) * p.ny / double(tiles_x * 32 * tiles_y * RLB_F32_BY);
        const bool linear = p.mapping == 2 || (p.mapping == 0 && fill < 0.97);
        if (linear) {
            block = dim3(32 * RLB_F32_BY, 1, 1);
            grid = dim3(unsigned((pairs + 32 * RLB_F32_BY - 1) / (32 * RLB_F32_BY)), 1, 1);
        } else {
            block = dim3(32, RLB_F32_BY, 1);
            grid = dim3(unsigned(tiles_x), unsigned(tiles_y), p.nz);
        }
    }
    const size_t smem = f32::step_smem_bytes(int(block.x * block.y), f32::kStageOn && VEC2 && !EULER, DIM);
    // the shared-memory limit is a per-device attribute of the kernel: set it
    // once per device and instantiation (a repeated set is harmless, so the
    // flags need no lock)
    constexpr int kMaxDevices = 64;
    static std::atomic<bool> attr_set[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= kMaxDevices || !attr_set[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(f32::step_f32_kernel<DIM, EULER, VEC2, LAT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        if (dev < kMaxDevices) attr_set[dev].store(true, std::memory_order_release);
    }
    f32::step_f32_kernel<DIM, EULER, VEC2, LAT><<<grid, block, smem, s>>>(p, f, h, fo, ho, prev);
    return cudaGetLastError();
}

template <bool EULER, bool VEC2, int LAT>
static cudaError_t launch_dim(const StepParams &p, int dim, const float *f, const float *h, float *fo,
                             float *ho, float *prev, cudaStream_t s)
{
    if (dim == 1) return launch_f32<1, EULER, VEC2, LAT>(p, f, h, fo, ho, prev, s);
    if (dim == 2) return launch_f32<2, EULER, VEC2, LAT>(p, f, h, fo, ho, prev, s);
    return launch_f32<3, EULER, VEC2, LAT>(p, f, h, fo, ho, prev, s);
}

template <int LAT>
static cudaError_t launch_lat(const StepParams &p, int dim, int euler, const float *f, const float *h,
                              float *fo, float *ho, float *prev, cudaStream_t s)
{
    // pair loads are 8-byte aligned when every row starts at an even index
    const bool vec = p.nx % 2 == 0;
    if (euler)
        return vec ? launch_dim<true, true, LAT>(p, dim, f, h, fo, ho, prev, s)
                   : launch_dim<true, false, LAT>(p, dim, f, h, fo, ho, prev, s);
    return vec ? launch_dim<false, true, LAT>(p, dim, f, h, fo, ho, prev, s)
               : launch_dim<false, false, LAT>(p, dim, f, h, fo, ho, prev, s);
}

cudaError_t launch_step_f32(const StepParams &p, int dim, int euler, const float *f, const float *h,
                            float *fo, float *ho, float *prev, cudaStream_t s)
{
    if (p.lat == 1) return launch_lat<1>(p, dim, euler, f, h, fo, ho, prev, s);
    return launch_lat<0>(p, dim, euler, f, h, fo, ho, prev, s);
}

}  // namespace rlb
