// The FP32-storage step with its Landau-frame recovery in FP64 (both time
// levels; rlb_options.recovery_fp64), in a unit of its own so that it
// compiles in parallel with the other step kernels.  Only the configuration
// it is measured on is instantiated: the extended lattice, the viscous step,
// 19 planes, even nx (aligned pair loads), tiles or the 1-D form; rlb_create
// rejects the others.
#include "rlb_step_f32_launch.cuh"

namespace rlb {

cudaError_t launch_step_f32_rec64(const StepParams &p, int dim, const float *f, const float *h, float *fo,
                                  float *ho, float *prev, cudaStream_t s)
{
    if (dim == 1) return launch_f32<1, false, true, 0, 19, false, true>(p, f, h, fo, ho, prev, s);
    if (dim == 2) return launch_f32<2, false, true, 0, 19, false, true>(p, f, h, fo, ho, prev, s);
    return launch_f32<3, false, true, 0, 19, false, true>(p, f, h, fo, ho, prev, s);
}

}  // namespace rlb
