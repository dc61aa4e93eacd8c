// Batched tubes: initialisation, macroscopic output and per-tube totals over
// the tube storage (packed fields in, packed fields out), and the dispatch of
// the persistent step kernel.
#include "rlb_cellops_f32.cuh"
#include "rlb_kernels.cuh"
#include "rlb_internal.h"

namespace rlb {
namespace batch {

cudaError_t launch_tubes(const Args &a, int threads, int bound, int cluster, cudaStream_t s,
                         int *nclusters_out)
{
    if (cluster < 1 || cluster > 8) return cudaErrorInvalidValue;
    if (cluster == 1) return launch_tubes_ca(a, threads, bound, s, nclusters_out);
    return launch_tubes_cg(a, threads, bound, cluster, s, nclusters_out);
}

// grid (ceil(max_nx / 256), B): cells x0 = 2 t and x0 + 1 of tube blockIdx.y
__global__ void tubes_init_kernel(const Tube *__restrict__ tubes, const long long *__restrict__ pack, long long ps,
                                  const double *__restrict__ n, const double *__restrict__ T,
                                  const double *__restrict__ ux, float *__restrict__ f, float *__restrict__ h,
                                  float *__restrict__ prev, unsigned *status)
{
    const int b = blockIdx.y;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const Tube t = tubes[b];
    if (x0 >= t.nx) return;
    const bool has1 = x0 + 1 < t.nx;
    const long long s0 = pack[b] + x0, d0 = (long long)t.off + x0;
    const f32::CellPair c{s0, has1 ? s0 + 1 : s0, d0, has1 ? d0 + 1 : d0, has1};
    f32::init_pair<0, false>(c, ps, n, T, ux, nullptr, nullptr, f, h, prev, status);
}

__global__ void tubes_macro_kernel(const Tube *__restrict__ tubes, const long long *__restrict__ pack,
                                   const int *__restrict__ par, long long ps, long long total,
                                   const float *__restrict__ f0, const float *__restrict__ h0,
                                   const float *__restrict__ f1, const float *__restrict__ h1,
                                   double *__restrict__ out, unsigned *status)
{
    const int b = blockIdx.y;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const Tube t = tubes[b];
    if (x0 >= t.nx) return;
    const bool has1 = x0 + 1 < t.nx;
    const bool one = par[b] != 0;
    const long long s0 = (long long)t.off + x0, d0 = pack[b] + x0;
    const f32::CellPair c{s0, has1 ? s0 + 1 : s0, d0, has1 ? d0 + 1 : d0, has1};
    f32::macro_pair<0, false>(c, ps, one ? f1 : f0, one ? h1 : h0, out, total, status);
}

// class of population i under the 1-D symmetry reduction, as the plane of
// its representative: rest, +x, -x, y/z axis, x+ diagonals, x- diagonals,
// y-z diagonals
__device__ __forceinline__ int class_plane(int i)
{
    if (i < 3) return i;
    if (i < 7) return 3;
    if (i >= 15) return 15;
    const int j = (i - 7) & 3;   // 7..10 and 11..14: signs (+,+) (+,-) (-,+) (-,-)
    return j < 2 ? 7 : 9;
}

__global__ void tubes_expand_kernel(const Tube *__restrict__ tubes, const int *__restrict__ par, long long ps,
                                    float *__restrict__ f0, float *__restrict__ h0, float *__restrict__ f1,
                                    float *__restrict__ h1)
{
    const int b = blockIdx.y;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const Tube t = tubes[b];
    if (x >= t.nx) return;
    const bool one = par[b] != 0;
    float *f = one ? f1 : f0, *h = one ? h1 : h0;
    const long long idx = (long long)t.off + x;
    for (int i = 3; i < 19; ++i) {
        const int r = class_plane(i);
        if (r == i) continue;
        f[i * ps + idx] = f[r * ps + idx];
        h[i * ps + idx] = h[r * ps + idx];
    }
}

// one block per tube, fixed reduction order (deterministic)
constexpr int kTubeTotBlock = 256;
__global__ void __launch_bounds__(kTubeTotBlock) tubes_totals_kernel(const Tube *__restrict__ tubes,
                                                                     const int *__restrict__ par, long long ps,
                                                                     const float *__restrict__ f0,
                                                                     const float *__restrict__ h0,
                                                                     const float *__restrict__ f1,
                                                                     const float *__restrict__ h1,
                                                                     double *__restrict__ out)
{
    const int b = blockIdx.x;
    const Tube t = tubes[b];
    const bool one = par[b] != 0;
    const float *f = one ? f1 : f0, *h = one ? h1 : h0;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int x = threadIdx.x; x < t.nx; x += blockDim.x) {
        const long long idx = (long long)t.off + x;
        for_pops(RLB_POPS, [&](auto ic) {
            constexpr int I = decltype(ic)::value;
            const double fv = double(f[I * ps + idx]);
            acc[0] += kXi0Sq * fv;
            if constexpr (cdir<I, 0>() != 0) acc[1] += kXi0 * double(cdir<I, 0>()) * fv;
            if constexpr (cdir<I, 1>() != 0) acc[2] += kXi0 * double(cdir<I, 1>()) * fv;
            if constexpr (cdir<I, 2>() != 0) acc[3] += kXi0 * double(cdir<I, 2>()) * fv;
            acc[4] += kXi0 * double(h[I * ps + idx]);
        });
    }
    __shared__ double sm[5][kTubeTotBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sm[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0.0;
        for (int w = 0; w < kTubeTotBlock / 32; ++w) v += sm[threadIdx.x][w];
        out[5 * (long long)b + threadIdx.x] = v;
    }
}

cudaError_t launch_tubes_init(int B, int max_nx, const Tube *tubes, const long long *pack, long long ps,
                              const double *n, const double *T, const double *ux, float *f, float *h,
                              float *prev, unsigned *status, cudaStream_t s)
{
    const dim3 grid((max_nx + 255) / 256, B, 1);
    tubes_init_kernel<<<grid, 128, 0, s>>>(tubes, pack, ps, n, T, ux, f, h, prev, status);
    return cudaGetLastError();
}

cudaError_t launch_tubes_macro(int B, int max_nx, const Tube *tubes, const long long *pack, const int *par,
                               long long ps, long long total, const float *f0, const float *h0,
                               const float *f1, const float *h1, double *out, unsigned *status,
                               cudaStream_t s)
{
    const dim3 grid((max_nx + 255) / 256, B, 1);
    tubes_macro_kernel<<<grid, 128, 0, s>>>(tubes, pack, par, ps, total, f0, h0, f1, h1, out, status);
    return cudaGetLastError();
}

cudaError_t launch_tubes_expand(int B, int max_nx, const Tube *tubes, const int *par, long long ps, float *f0,
                                float *h0, float *f1, float *h1, cudaStream_t s)
{
    const dim3 grid((max_nx + 127) / 128, B, 1);
    tubes_expand_kernel<<<grid, 128, 0, s>>>(tubes, par, ps, f0, h0, f1, h1);
    return cudaGetLastError();
}

cudaError_t launch_tubes_totals(int B, const Tube *tubes, const int *par, long long ps, const float *f0,
                                const float *h0, const float *f1, const float *h1, double *out,
                                cudaStream_t s)
{
    tubes_totals_kernel<<<B, kTubeTotBlock, 0, s>>>(tubes, par, ps, f0, h0, f1, h1, out);
    return cudaGetLastError();
}

}  // namespace batch
}  // namespace rlb
