// FP64 form of the fused step: populations stored and computed in double.
#include "rlb_step_impl.cuh"

namespace rlb {
cudaError_t launch_step_f64(const StepParams &p, int dim, int euler, const double *f,
                            const double *h, double *fo, double *ho, double *prev, cudaStream_t s)
{
    return launch_step_any<double>(p, dim, euler, f, h, fo, ho, prev, s);
}

// the kernel launch_step_np picks (the same decisions, without launching)
const char *f64_step_kernel_name(const StepParams &p, int dim)
{
    const long long cells = (long long)p.nx * p.ny * p.nz;
    if (cells < 128LL * sm_count() && p.mapping != 1 && p.mapping != 3) return "fp64_small";
    if (dim == 1) return "fp64_1d";
    const long long tiles_x = (p.nx + 31) / 32, tiles_y = (p.ny + 3) / 4;
    const double fill = double(p.nx) * p.ny / double(tiles_x * 32 * tiles_y * 4);
    return (p.mapping == 2 || (p.mapping == 0 && fill < 0.97)) ? "fp64_linear" : "fp64_tiles";
}
}  // namespace rlb
