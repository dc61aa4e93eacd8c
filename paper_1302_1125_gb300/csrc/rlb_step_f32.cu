// FP32-storage form of the fused step (see rlb_step_f32.cuh): populations
// stored, streamed and relaxed in float, two cells per thread, double-float
// moment sums, no FP64 instructions.  This unit holds the tiled
// instantiations and the 1-D form; rlb_step_f32_lin.cu the linear mapping.
#include "rlb_step_f32_launch.cuh"

namespace rlb {

cudaError_t launch_step_f32(const StepParams &p, int dim, int euler, const float *f, const float *h,
                            float *fo, float *ho, float *prev, cudaStream_t s, const TileMaps *maps)
{
    if (maps && f32_bulk_eligible(p, dim, euler)) return launch_step_f32_bulk(p, f, h, fo, ho, prev, maps, s);
    if (f32_use_linear(p, dim)) return launch_step_f32_linear(p, dim, euler, f, h, fo, ho, prev, s);
    return launch_f32_mapped<false>(p, dim, euler, f, h, fo, ho, prev, s);
}

// One z-plane of a slab (the f and h planes of its block rows) about this
// size: the slab's planes that the z-stencils of the resident blocks read
// then stay in L2 (measured on the 512 x 256 x 256 grid: 16 block rows,
// 10 MB, the fastest of 4, 8, 16 and all 32)
#ifndef RLB_SLAB_TARGET_KB
#define RLB_SLAB_TARGET_KB 10240
#endif
int f32_slab_rows(int nx, int ny)
{
    const double row_bytes = double(RLB_F32_BY) * double(nx) * 38.0 * sizeof(float);
    const int nby = (ny + RLB_F32_BY - 1) / RLB_F32_BY;
    const int s = int(double(RLB_SLAB_TARGET_KB) * 1024.0 / row_bytes);
    return s < 1 ? 1 : (s > nby ? nby : s);
}

const char *f32_step_kernel_name(const StepParams &p, int dim, int euler, bool have_maps)
{
    if (have_maps && f32_bulk_eligible(p, dim, euler)) return "fp32_bulk_tiles";
    if (f32_use_linear(p, dim)) return "fp32_linear";
    return dim == 1 ? "fp32_1d" : "fp32_tiles";
}

}  // namespace rlb
