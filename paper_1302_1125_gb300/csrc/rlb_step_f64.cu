// FP64 form of the fused step: populations stored and computed in double.
#include "rlb_step_impl.cuh"

namespace rlb {
cudaError_t launch_step_f64(const StepParams &p, int dim, int euler, const double *f,
                            const double *h, double *fo, double *ho, double *prev, cudaStream_t s)
{
    return launch_step_any<double>(p, dim, euler, f, h, fo, ho, prev, s);
}
}  // namespace rlb
