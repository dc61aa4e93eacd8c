// The FP32-storage step kernel under the linear thread mapping (grids of 2
// or 3 dimensions whose nx does not fill the 64-cell-wide tiles), in a unit
// of its own so that it compiles in parallel with rlb_step_f32.cu.
#include "rlb_step_f32_launch.cuh"

namespace rlb {

cudaError_t launch_step_f32_linear(const StepParams &p, int dim, int euler, const float *f, const float *h,
                                   float *fo, float *ho, float *prev, cudaStream_t s)
{
    return launch_f32_mapped<true>(p, dim, euler, f, h, fo, ho, prev, s);
}

}  // namespace rlb
