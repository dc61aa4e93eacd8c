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

const char *f32_step_kernel_name(const StepParams &p, int dim, int euler, bool have_maps)
{
    if (have_maps && f32_bulk_eligible(p, dim, euler)) return "fp32_bulk_tiles";
    if (f32_use_linear(p, dim)) return "fp32_linear";
    return dim == 1 ? "fp32_1d" : "fp32_tiles";
}

}  // namespace rlb
