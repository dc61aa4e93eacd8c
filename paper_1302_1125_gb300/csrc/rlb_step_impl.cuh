// rlb_step_impl.cuh -- launch configuration of the fused step kernel, shared
// by the FP64 and FP32-storage translation units.
#pragma once

#include "rlb_kernels.cuh"

namespace rlb {

template <typename T, int DIM, bool EULER, int LAT>
cudaError_t launch_step_t(const StepParams &p, const T *f, const T *h, T *fo, T *ho, T *prev,
                          cudaStream_t s)
{
    if (DIM == 1) {
        step_kernel<T, DIM, EULER, LAT><<<(p.nx + 127) / 128, 128, 0, s>>>(p, f, h, fo, ho, prev);
        return cudaGetLastError();
    }
    // tiles of 32 x 4 cells when nx and ny fill them, else 128 consecutive
    // cells of the x-fastest order per block
    const long long tiles_x = (p.nx + 31) / 32, tiles_y = (p.ny + 3) / 4;
    const long long cells = (long long)p.nx * p.ny * p.nz;
    const double fill = double(p.nx) * p.ny / double(tiles_x * 32 * tiles_y * 4);
    if (p.mapping == 2 || (p.mapping == 0 && fill < 0.97)) {
        step_kernel<T, DIM, EULER, LAT, true><<<unsigned((cells + 127) / 128), 128, 0, s>>>(p, f, h, fo, ho, prev);
    } else {
        const dim3 grid(unsigned(tiles_x), unsigned(tiles_y), p.nz);
        step_kernel<T, DIM, EULER, LAT, false><<<grid, dim3(32, 4, 1), 0, s>>>(p, f, h, fo, ho, prev);
    }
    return cudaGetLastError();
}

template <typename T, int LAT>
cudaError_t launch_step_lat(const StepParams &p, int dim, int euler, const T *f, const T *h, T *fo, T *ho,
                            T *prev, cudaStream_t s)
{
    if (euler) {
        if (dim == 1) return launch_step_t<T, 1, true, LAT>(p, f, h, fo, ho, prev, s);
        if (dim == 2) return launch_step_t<T, 2, true, LAT>(p, f, h, fo, ho, prev, s);
        return launch_step_t<T, 3, true, LAT>(p, f, h, fo, ho, prev, s);
    }
    if (dim == 1) return launch_step_t<T, 1, false, LAT>(p, f, h, fo, ho, prev, s);
    if (dim == 2) return launch_step_t<T, 2, false, LAT>(p, f, h, fo, ho, prev, s);
    return launch_step_t<T, 3, false, LAT>(p, f, h, fo, ho, prev, s);
}

template <typename T>
cudaError_t launch_step_any(const StepParams &p, int dim, int euler, const T *f, const T *h, T *fo,
                            T *ho, T *prev, cudaStream_t s)
{
    if (p.lat == 1) return launch_step_lat<T, 1>(p, dim, euler, f, h, fo, ho, prev, s);
    return launch_step_lat<T, 0>(p, dim, euler, f, h, fo, ho, prev, s);
}

}  // namespace rlb
