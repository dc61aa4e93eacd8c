// rlb_step_impl.cuh -- launch configuration of the fused step kernel, shared
// by the FP64 and FP32-storage translation units.
#pragma once

#include "rlb_kernels.cuh"

namespace rlb {

template <typename T, int DIM, bool EULER>
cudaError_t launch_step_t(const StepParams &p, const T *f, const T *h, T *fo, T *ho, T *prev,
                          cudaStream_t s)
{
    dim3 block, grid;
    if (DIM == 1) {
        block = dim3(128, 1, 1);
        grid = dim3((p.nx + 127) / 128, 1, 1);
    } else {
        block = dim3(32, 4, 1);
        grid = dim3((p.nx + 31) / 32, (p.ny + 3) / 4, p.nz);
    }
    step_kernel<T, DIM, EULER><<<grid, block, 0, s>>>(p, f, h, fo, ho, prev);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step_any(const StepParams &p, int dim, int euler, const T *f, const T *h, T *fo,
                            T *ho, T *prev, cudaStream_t s)
{
    if (euler) {
        if (dim == 1) return launch_step_t<T, 1, true>(p, f, h, fo, ho, prev, s);
        if (dim == 2) return launch_step_t<T, 2, true>(p, f, h, fo, ho, prev, s);
        return launch_step_t<T, 3, true>(p, f, h, fo, ho, prev, s);
    }
    if (dim == 1) return launch_step_t<T, 1, false>(p, f, h, fo, ho, prev, s);
    if (dim == 2) return launch_step_t<T, 2, false>(p, f, h, fo, ho, prev, s);
    return launch_step_t<T, 3, false>(p, f, h, fo, ho, prev, s);
}

}  // namespace rlb
