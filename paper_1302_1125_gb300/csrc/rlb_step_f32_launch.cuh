// rlb_step_f32_launch.cuh -- launch configuration of the FP32-storage step
// kernel, shared by the two translation units that instantiate it (tiles:
// rlb_step_f32.cu; the linear mapping: rlb_step_f32_lin.cu, compiled in
// parallel).
#pragma once

#include <atomic>

#include "rlb_step_f32.cuh"

namespace rlb {

// grids of 2 or 3 dimensions: the linear mapping when forced, or when the
// 64 x BY-cell tiles would leave more than 3 % of their lanes idle
inline bool f32_use_linear(const StepParams &p, int dim)
{
    if (dim == 1 || p.mapping == 1 || p.mapping == 3) return false;   // 3: tiles (bulk-staged where eligible)
    if (p.mapping == 2) return true;
    const long long npairs = (p.nx + 1) / 2;
    const long long tiles_x = (npairs + 31) / 32, tiles_y = (p.ny + RLB_F32_BY - 1) / RLB_F32_BY;
    const double fill = double(npairs) * p.ny / double(tiles_x * 32 * tiles_y * RLB_F32_BY);
    return fill < 0.97;
}

template <int DIM, bool EULER, bool VEC2, int LAT, int NP, bool LIN, bool REC64 = false>
cudaError_t launch_f32(const StepParams &p, const float *f, const float *h, float *fo, float *ho, float *prev,
                       cudaStream_t s)
{
    if constexpr (DIM == 2 && !EULER && NP == 19 && !REC64) {
        if (p.sym == 2) return launch_f32<2, false, VEC2, LAT, 14, LIN>(p, f, h, fo, ho, prev, s);
    }
    if constexpr (DIM == 1 && !EULER && NP == 19 && !LIN && !REC64) {
        if (p.sym == 1) return launch_f32<1, false, VEC2, LAT, 7, false>(p, f, h, fo, ho, prev, s);
    }
    const int npairs = (p.nx + 1) / 2;
    dim3 block, grid;
    if (LIN) {
        // 32 BY consecutive pairs of the x-fastest order per block
        const long long pairs = (long long)npairs * p.ny * p.nz;
        block = dim3(32 * RLB_F32_BY, 1, 1);
        grid = dim3(unsigned((pairs + 32 * RLB_F32_BY - 1) / (32 * RLB_F32_BY)), 1, 1);
    } else if (DIM == 1) {
        block = dim3(128, 1, 1);
        grid = dim3((npairs + 127) / 128, 1, 1);
    } else {
        // 32 x 8 threads (64 x 8 cells), two blocks per SM at <= 128 registers:
        // the best of a sweep over block shapes and register caps on GB300
        block = dim3(32, RLB_F32_BY, 1);
        grid = dim3((npairs + 31) / 32, (p.ny + RLB_F32_BY - 1) / RLB_F32_BY, p.nz);
    }
    const size_t smem = f32::step_smem_bytes(int(block.x * block.y), f32::kStageOn && VEC2 && !EULER, DIM);
    // the shared-memory limit is a per-device attribute of the kernel: set it
    // once per device and instantiation (a repeated set is harmless, so the
    // flags need no lock)
    constexpr int kMaxDevices = 64;
    static std::atomic<bool> attr_set[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= kMaxDevices || !attr_set[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(f32::step_f32_kernel<DIM, EULER, VEC2, LAT, NP, LIN, REC64>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        if (dev < kMaxDevices) attr_set[dev].store(true, std::memory_order_release);
    }
    f32::step_f32_kernel<DIM, EULER, VEC2, LAT, NP, LIN, REC64><<<grid, block, smem, s>>>(p, f, h, fo, ho, prev);
    return cudaGetLastError();
}

// dim 2 or 3 (and 1 when !LIN), Euler or viscous, lattice from p.lat
template <bool LIN>
cudaError_t launch_f32_mapped(const StepParams &p, int dim, int euler, const float *f, const float *h, float *fo,
                              float *ho, float *prev, cudaStream_t s)
{
    auto go = [&](auto lc, auto ec, auto vc) -> cudaError_t {
        constexpr int L = decltype(lc)::value;
        constexpr bool E = decltype(ec)::value, V = decltype(vc)::value;
        if constexpr (!LIN) {
            if (dim == 1) return launch_f32<1, E, V, L, 19, false>(p, f, h, fo, ho, prev, s);
        }
        if (dim == 2) return launch_f32<2, E, V, L, 19, LIN>(p, f, h, fo, ho, prev, s);
        return launch_f32<3, E, V, L, 19, LIN>(p, f, h, fo, ho, prev, s);
    };
    // pair loads are 8-byte aligned when every row starts at an even index
    const bool vec = p.nx % 2 == 0;
    auto by_lat = [&](auto ec, auto vc) {
        return p.lat == 1 ? go(std::integral_constant<int, 1>{}, ec, vc)
                          : go(std::integral_constant<int, 0>{}, ec, vc);
    };
    auto by_vec = [&](auto ec) {
        return vec ? by_lat(ec, std::true_type{}) : by_lat(ec, std::false_type{});
    };
    return euler ? by_vec(std::true_type{}) : by_vec(std::false_type{});
}

// the linear instantiations (rlb_step_f32_lin.cu)
cudaError_t launch_step_f32_linear(const StepParams &p, int dim, int euler, const float *f, const float *h,
                                   float *fo, float *ho, float *prev, cudaStream_t s);

}  // namespace rlb
