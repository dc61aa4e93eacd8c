// Initialisation, macroscopic output and conserved-total kernels.
#include <utility>

#include "rlb_cellops.cuh"
#include "rlb_cellops_f32.cuh"

namespace rlb {

// (sym: the state must have u_y = u_z = 0 for the 1-D symmetry reduction,
// u_z = 0 for the 2-D one)
template <typename T, int LAT>
__global__ void init_kernel(int N, long long ps, const double *__restrict__ n,
                            const double *__restrict__ Tt, const double *__restrict__ ux,
                            const double *__restrict__ uy, const double *__restrict__ uz,
                            T *__restrict__ f, T *__restrict__ h, T *__restrict__ prev,
                            unsigned *status, int sym)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N) return;
    if (sym && (uz[idx] != 0.0 || (sym == 1 && uy[idx] != 0.0))) atomicOr(status, unsigned(ST_ASYMMETRIC));
    init_cell<T, LAT>(idx, idx, ps, n, Tt, ux, uy, uz, f, h, prev, status);
}

// moments + recovery of the current populations: n, e, u_x, u_y, u_z, gamma
template <typename T, int LAT>
__global__ void macro_kernel(int N, long long ps, const T *__restrict__ f,
                             const T *__restrict__ h, double *__restrict__ out,
                             unsigned *status)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N) return;
    macro_cell<T, LAT>(idx, ps, f, h, out, idx, N, status);
}

// solid cells: the equilibrium of st = {n, T, 0} (the same code as the
// initialisation, so a solid cell holds what rlb_init writes for that state)
template <typename T, int LAT>
__global__ void solid_reset_kernel(int M, const int *__restrict__ idx, long long ps, const double *__restrict__ st,
                                   T *__restrict__ f, T *__restrict__ h, T *__restrict__ prev, unsigned *status)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    init_cell<T, LAT>(0, idx[j], ps, st, st + 1, st + 2, st + 2, st + 2, f, h, prev, status);
}

// FP32-storage forms of the three kernels above, two cells per thread in
// float arithmetic (rlb_cellops_f32.cuh): consecutive cells i0 = 2 t, i0 + 1
// (sym: the state must have u_y = u_z = 0 for the 1-D symmetry reduction,
// u_z = 0 for the 2-D one)
template <int LAT>
__global__ void init_kernel_f32(int N, long long ps, const double *__restrict__ n, const double *__restrict__ Tt,
                                const double *__restrict__ ux, const double *__restrict__ uy,
                                const double *__restrict__ uz, float *__restrict__ f, float *__restrict__ h,
                                float *__restrict__ prev, unsigned *status, int sym)
{
    const long long i0 = 2LL * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 >= N) return;
    const bool has1 = i0 + 1 < N;
    const long long i1 = has1 ? i0 + 1 : i0;
    if (sym && (uz[i0] != 0.0 || uz[i1] != 0.0 || (sym == 1 && (uy[i0] != 0.0 || uy[i1] != 0.0))))
        atomicOr(status, unsigned(ST_ASYMMETRIC));
    f32::init_pair<LAT, true>(f32::CellPair{i0, i1, i0, i1, has1}, ps, n, Tt, ux, uy, uz, f, h, prev, status);
}

// the members of the reductions' classes: population kMember[j][1] equals
// its class representative kMember[j][0].  2-D (the first 5): mirror images
// in z.  1-D (all 12): the y/z axis populations, the diagonals with
// c_x = +2, those with c_x = -2, the y-z diagonals (the classes of the
// batched-tube reduction).
__constant__ int kMember[2][12][2] = {
    {{3, 4}, {3, 5}, {3, 6}, {7, 8}, {7, 11}, {7, 12}, {9, 10}, {9, 13}, {9, 14}, {15, 16}, {15, 17}, {15, 18}},
    {{5, 6}, {11, 12}, {13, 14}, {15, 16}, {17, 18}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}}};

template <typename T>
__global__ void sym_kernel(int expand, int sym, int N, long long ps, T *__restrict__ f, T *__restrict__ h,
                           T *__restrict__ prev, unsigned *status)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int t = sym == 1 ? 0 : 1, m = sym == 1 ? 12 : 5;
    bool same = true;
    for (int j = 0; j < m; ++j) {
        const long long a = kMember[t][j][0] * ps + i, b = kMember[t][j][1] * ps + i;
        if (expand) {
            f[b] = f[a];
            h[b] = h[a];
        } else {
            same = same && f[b] == f[a] && h[b] == h[a];
        }
    }
    // the FP32-storage form's previous level holds raw sums (sum c_y f and
    // sum c_z f vanish); the FP64 form's holds u' (u'_y and u'_z are zero)
    if (expand) {
        if (sym == 1) prev[2 * ps + i] = T(0);
        prev[3 * ps + i] = T(0);
    } else if (!same) {
        atomicOr(status, unsigned(ST_ASYMMETRIC));
    }
}

template <int LAT>
__global__ void macro_kernel_f32(int N, long long ps, const float *__restrict__ f, const float *__restrict__ h,
                                 double *__restrict__ out, unsigned *status)
{
    const long long i0 = 2LL * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 >= N) return;
    const bool has1 = i0 + 1 < N;
    const long long i1 = has1 ? i0 + 1 : i0;
    f32::macro_pair<LAT, true>(f32::CellPair{i0, i1, i0, i1, has1}, ps, f, h, out, N, status);
}

// solid cells idx[2 t] and idx[2 t + 1], both from the state st = {n, T, 0}
template <int LAT>
__global__ void solid_reset_kernel_f32(int M, const int *__restrict__ idx, long long ps,
                                       const double *__restrict__ st, float *__restrict__ f, float *__restrict__ h,
                                       float *__restrict__ prev, unsigned *status)
{
    const int j = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (j >= M) return;
    const bool has1 = j + 1 < M;
    const long long d0 = idx[j], d1 = has1 ? idx[j + 1] : d0;
    f32::init_pair<LAT, false>(f32::CellPair{0, 0, d0, d1, has1}, ps, st, st + 1, st + 2, st + 2, st + 2, f, h,
                               prev, status);
}

// per-block partial sums of (T^00, T^0x, T^0y, T^0z, N^0); fixed grid and
// fixed reduction order, so the result is deterministic
constexpr int kTotBlock = 256;
template <typename T, int LAT>
__global__ void __launch_bounds__(kTotBlock) totals_kernel(int N, long long ps,
                                                           const T *__restrict__ f,
                                                           const T *__restrict__ h,
                                                           double *__restrict__ partial)
{
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
        for_pops(RLB_POPS, [&](auto ic) {
            constexpr int I = decltype(ic)::value;
            const double fv = double(f[I * ps + idx]);
            acc[0] += Lat<LAT>::xi0sq * fv;
            if constexpr (cdir<I, 0, LAT>() != 0) acc[1] += Lat<LAT>::xi0 * double(cdir<I, 0, LAT>()) * fv;
            if constexpr (cdir<I, 1, LAT>() != 0) acc[2] += Lat<LAT>::xi0 * double(cdir<I, 1, LAT>()) * fv;
            if constexpr (cdir<I, 2, LAT>() != 0) acc[3] += Lat<LAT>::xi0 * double(cdir<I, 2, LAT>()) * fv;
            acc[4] += Lat<LAT>::xi0 * double(h[I * ps + idx]);
        });
    }
    __shared__ double sm[5][kTotBlock / 32];
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
        for (int w = 0; w < kTotBlock / 32; ++w) v += sm[threadIdx.x][w];
        partial[blockIdx.x * 5 + threadIdx.x] = v;
    }
}

__global__ void totals_finish(int nblocks, const double *__restrict__ partial, double *out)
{
    if (threadIdx.x < 5) {
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += partial[b * 5 + threadIdx.x];
        out[threadIdx.x] = v;
    }
}


cudaError_t launch_sym(int fp32, int expand, int sym, int N, long long ps, void *f, void *h, void *prev,
                       unsigned *status, cudaStream_t s)
{
    if (sym != 1 && sym != 2) return cudaErrorInvalidValue;
    const int b = 256, g = (N + b - 1) / b;
    if (fp32)
        sym_kernel<float><<<g, b, 0, s>>>(expand, sym, N, ps, (float *)f, (float *)h, (float *)prev, status);
    else
        sym_kernel<double><<<g, b, 0, s>>>(expand, sym, N, ps, (double *)f, (double *)h, (double *)prev, status);
    return cudaGetLastError();
}

cudaError_t launch_init(int fp32, int N, long long ps, const double *n, const double *T,
                        const double *ux, const double *uy, const double *uz, void *f, void *h,
                        void *prev, unsigned *status, cudaStream_t s, int lat, int sym)
{
    const int b = 128, g = (N + b - 1) / b, g2 = (N + 2 * b - 1) / (2 * b);
    auto go = [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        if (fp32)
            init_kernel_f32<L><<<g2, b, 0, s>>>(N, ps, n, T, ux, uy, uz, (float *)f, (float *)h, (float *)prev,
                                                status, sym);
        else
            init_kernel<double, L><<<g, b, 0, s>>>(N, ps, n, T, ux, uy, uz, (double *)f, (double *)h,
                                                   (double *)prev, status, sym);
    };
    if (lat == 1) go(std::integral_constant<int, 1>{});
    else go(std::integral_constant<int, 0>{});
    return cudaGetLastError();
}

cudaError_t launch_macro(int fp32, int N, long long ps, const void *f, const void *h, double *out,
                         unsigned *status, cudaStream_t s, int lat)
{
    const int b = 128, g = (N + b - 1) / b, g2 = (N + 2 * b - 1) / (2 * b);
    auto go = [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        if (fp32)
            macro_kernel_f32<L><<<g2, b, 0, s>>>(N, ps, (const float *)f, (const float *)h, out, status);
        else
            macro_kernel<double, L><<<g, b, 0, s>>>(N, ps, (const double *)f, (const double *)h, out,
                                                    status);
    };
    if (lat == 1) go(std::integral_constant<int, 1>{});
    else go(std::integral_constant<int, 0>{});
    return cudaGetLastError();
}

cudaError_t launch_solid_reset(int fp32, int M, const int *idx, long long ps, const double *st, void *f,
                               void *h, void *prev, unsigned *status, cudaStream_t s, int lat)
{
    const int b = 128, g = (M + b - 1) / b, g2 = (M + 2 * b - 1) / (2 * b);
    auto go = [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        if (fp32)
            solid_reset_kernel_f32<L><<<g2, b, 0, s>>>(M, idx, ps, st, (float *)f, (float *)h, (float *)prev,
                                                       status);
        else
            solid_reset_kernel<double, L><<<g, b, 0, s>>>(M, idx, ps, st, (double *)f, (double *)h,
                                                          (double *)prev, status);
    };
    if (lat == 1) go(std::integral_constant<int, 1>{});
    else go(std::integral_constant<int, 0>{});
    return cudaGetLastError();
}

int totals_blocks(int N)
{
    const int want = (N + kTotBlock - 1) / kTotBlock;
    return want < 1 ? 1 : (want > 1216 ? 1216 : want);   // 1216 = 8 x 152 SMs
}

cudaError_t launch_totals(int fp32, int N, long long ps, const void *f, const void *h,
                          double *partial, double *out, cudaStream_t s, int lat)
{
    const int nb = totals_blocks(N);
    auto go = [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        if (fp32)
            totals_kernel<float, L><<<nb, kTotBlock, 0, s>>>(N, ps, (const float *)f, (const float *)h, partial);
        else
            totals_kernel<double, L><<<nb, kTotBlock, 0, s>>>(N, ps, (const double *)f, (const double *)h,
                                                             partial);
    };
    if (lat == 1) go(std::integral_constant<int, 1>{});
    else go(std::integral_constant<int, 0>{});
    totals_finish<<<1, 32, 0, s>>>(nb, partial, out);
    return cudaGetLastError();
}

}  // namespace rlb
