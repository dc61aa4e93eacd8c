// rlb_step_impl.cuh -- launch configuration of the fused step kernel, shared
// by the FP64 and FP32-storage translation units.
#pragma once

#include "rlb_kernels.cuh"

namespace rlb {

// SMs of the current device (looked up once per device)
inline int sm_count()
{
    constexpr int kMaxDevices = 64;
    static int cache[kMaxDevices] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev < kMaxDevices && cache[dev] > 0) return cache[dev];
    int n = 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    if (dev < kMaxDevices) cache[dev] = n;
    return n;
}

template <typename T, int DIM, bool EULER, int LAT, int NP>
cudaError_t launch_step_np(const StepParams &p, const T *f, const T *h, T *fo, T *ho, T *prev,
                          cudaStream_t s)
{
    const long long cells = (long long)p.nx * p.ny * p.nz;
    // Grids with fewer cells than one block of 128 per SM: blocks of one to
    // four warps of consecutive cells (x-fastest order) spread the cells over
    // more SMs.  Measured: steps 6 % shorter on 800- to 8192-cell tubes and
    // 32 x 16 x 16 grids.  The step time of such grids stays set by one
    // warp's FP64 instructions at one scheduler's FP64 rate.
    const int nsm = sm_count();
    if (cells < 128LL * nsm && p.mapping != 1 && p.mapping != 3) {   // 3: tiles (FP32: bulk-staged)
        int bs = int(((cells + nsm - 1) / nsm + 31) / 32 * 32);
        bs = bs < 32 ? 32 : (bs > 128 ? 128 : bs);
        const unsigned nb = unsigned((cells + bs - 1) / bs);
        if constexpr (DIM == 1) step_kernel<T, DIM, EULER, LAT, false, NP><<<nb, bs, 0, s>>>(p, f, h, fo, ho, prev);
        else step_kernel<T, DIM, EULER, LAT, true, NP><<<nb, bs, 0, s>>>(p, f, h, fo, ho, prev);
        return cudaGetLastError();
    }
    if constexpr (DIM == 1) {
        step_kernel<T, DIM, EULER, LAT, false, NP><<<(p.nx + 127) / 128, 128, 0, s>>>(p, f, h, fo, ho, prev);
    } else {
        // tiles of 32 x 4 cells when nx and ny fill them, else 128 consecutive
        // cells of the x-fastest order per block
        const long long tiles_x = (p.nx + 31) / 32, tiles_y = (p.ny + 3) / 4;
        const double fill = double(p.nx) * p.ny / double(tiles_x * 32 * tiles_y * 4);
        if (p.mapping == 2 || (p.mapping == 0 && fill < 0.97)) {
            step_kernel<T, DIM, EULER, LAT, true, NP><<<unsigned((cells + 127) / 128), 128, 0, s>>>(p, f, h, fo, ho,
                                                                                                    prev);
        } else {
            const dim3 grid(unsigned(tiles_x), unsigned(tiles_y), p.nz);
            step_kernel<T, DIM, EULER, LAT, false, NP><<<grid, dim3(32, 4, 1), 0, s>>>(p, f, h, fo, ho, prev);
        }
    }
    return cudaGetLastError();
}

// the symmetry reductions (p.sym: 1 on 1-D grids, 2 on 2-D grids; viscous)
template <typename T, int DIM, bool EULER, int LAT>
cudaError_t launch_step_t(const StepParams &p, const T *f, const T *h, T *fo, T *ho, T *prev,
                          cudaStream_t s)
{
    if constexpr (DIM == 1 && !EULER) {
        if (p.sym == 1) return launch_step_np<T, 1, false, LAT, 7>(p, f, h, fo, ho, prev, s);
    }
    if constexpr (DIM == 2 && !EULER) {
        if (p.sym == 2) return launch_step_np<T, 2, false, LAT, 14>(p, f, h, fo, ho, prev, s);
    }
    return launch_step_np<T, DIM, EULER, LAT, 19>(p, f, h, fo, ho, prev, s);
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
