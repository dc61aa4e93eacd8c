// FP32-storage form of the fused step: populations stored and streamed in
// float; moment sums, the Landau-frame recovery and the equilibrium
// coefficients in double.
#include "rlb_step_impl.cuh"

namespace rlb {
cudaError_t launch_step_f32(const StepParams &p, int dim, int euler, const float *f,
                            const float *h, float *fo, float *ho, float *prev, cudaStream_t s)
{
    return launch_step_any<float>(p, dim, euler, f, h, fo, ho, prev, s);
}
}  // namespace rlb
