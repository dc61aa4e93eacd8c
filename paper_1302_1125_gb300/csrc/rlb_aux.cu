// Initialisation, macroscopic output and conserved-total kernels.
#include "rlb_kernels.cuh"

namespace rlb {

// f = f^eq(P = nT, u), h = h^eq(n, u), previous level = this state
template <typename T>
__global__ void init_kernel(int N, long long ps, const double *__restrict__ n,
                            const double *__restrict__ Tt, const double *__restrict__ ux,
                            const double *__restrict__ uy, const double *__restrict__ uz,
                            T *__restrict__ f, T *__restrict__ h, T *__restrict__ prev,
                            unsigned *status)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N) return;
    const double vx = ux[idx], vy = uy[idx], vz = uz[idx];
    const double v2 = vx * vx + vy * vy + vz * vz;
    const double g = 1.0 / sqrt(1.0 - v2);
    if (!(n[idx] > 0.0 && Tt[idx] > 0.0 && v2 < 1.0 && isfinite(n[idx] * Tt[idx]) && isfinite(g)))
        atomicOr(status, unsigned(ST_NONPHYSICAL));
    Macro m;
    m.P = n[idx] * Tt[idx];
    m.ux = g * vx;
    m.uy = g * vy;
    m.uz = g * vz;
    m.n = n[idx];
    Coef<double> a;
    coef_f(m, a);
    const EqW<T> kf = weigh_f<T>(a);
    coef_h(m, a);
    const EqW<T> kh = weigh_h<T>(a);
    double S = 0.0, Vx = 0.0, Vy = 0.0, Vz = 0.0, Sh = 0.0;
    for_pops(RLB_POPS, [&](auto ic) {
        constexpr int I = decltype(ic)::value;
        const T fv = eq_pop<I>(kf), hv = eq_pop<I>(kh);
        f[I * ps + idx] = fv;
        h[I * ps + idx] = hv;
        S += double(fv);
        Sh += double(hv);
        if constexpr (cdir<I, 0>() != 0) Vx += double(cdir<I, 0>()) * double(fv);
        if constexpr (cdir<I, 1>() != 0) Vy += double(cdir<I, 1>()) * double(fv);
        if constexpr (cdir<I, 2>() != 0) Vz += double(cdir<I, 2>()) * double(fv);
    });
    if constexpr (sizeof(T) == 4) {
        // FP32-storage form: the previous level is the raw moment sums
        prev[0 * ps + idx] = T(S);
        prev[1 * ps + idx] = T(Vx);
        prev[2 * ps + idx] = T(Vy);
        prev[3 * ps + idx] = T(Vz);
        prev[4 * ps + idx] = T(Sh);
    } else {
        prev[0 * ps + idx] = T(m.P);
        prev[1 * ps + idx] = T(m.ux);
        prev[2 * ps + idx] = T(m.uy);
        prev[3 * ps + idx] = T(m.uz);
        prev[4 * ps + idx] = T(m.n);
    }
}

// moments + recovery of the current populations: n, e, u_x, u_y, u_z, gamma
template <typename T>
__global__ void macro_kernel(int N, long long ps, const T *__restrict__ f,
                             const T *__restrict__ h, double *__restrict__ out,
                             unsigned *status)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N) return;
    double sf = 0.0, sh = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    for_pops(RLB_POPS, [&](auto ic) {
        constexpr int I = decltype(ic)::value;
        const double fv = double(f[I * ps + idx]);
        sf += fv;
        sh += double(h[I * ps + idx]);
        if constexpr (cdir<I, 0>() != 0) mx += double(cdir<I, 0>()) * fv;
        if constexpr (cdir<I, 1>() != 0) my += double(cdir<I, 1>()) * fv;
        if constexpr (cdir<I, 2>() != 0) mz += double(cdir<I, 2>()) * fv;
    });
    Macro m;
    if (!recover(kXi0Sq * sf, kXi0 * mx, kXi0 * my, kXi0 * mz, kXi0 * sh, m))
        atomicOr(status, unsigned(ST_NONPHYSICAL));
    const double g = sqrt(1.0 + m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
    out[0 * (long long)N + idx] = m.n;
    out[1 * (long long)N + idx] = 3.0 * m.P;
    out[2 * (long long)N + idx] = m.ux / g;
    out[3 * (long long)N + idx] = m.uy / g;
    out[4 * (long long)N + idx] = m.uz / g;
    out[5 * (long long)N + idx] = g;
}

// per-block partial sums of (T^00, T^0x, T^0y, T^0z, N^0); fixed grid and
// fixed reduction order, so the result is deterministic
constexpr int kTotBlock = 256;
template <typename T>
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
            acc[0] += kXi0Sq * fv;
            if constexpr (cdir<I, 0>() != 0) acc[1] += kXi0 * double(cdir<I, 0>()) * fv;
            if constexpr (cdir<I, 1>() != 0) acc[2] += kXi0 * double(cdir<I, 1>()) * fv;
            if constexpr (cdir<I, 2>() != 0) acc[3] += kXi0 * double(cdir<I, 2>()) * fv;
            acc[4] += kXi0 * double(h[I * ps + idx]);
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


cudaError_t launch_init(int fp32, int N, long long ps, const double *n, const double *T,
                        const double *ux, const double *uy, const double *uz, void *f, void *h,
                        void *prev, unsigned *status, cudaStream_t s)
{
    const int b = 128, g = (N + b - 1) / b;
    if (fp32)
        init_kernel<float><<<g, b, 0, s>>>(N, ps, n, T, ux, uy, uz, (float *)f, (float *)h,
                                           (float *)prev, status);
    else
        init_kernel<double><<<g, b, 0, s>>>(N, ps, n, T, ux, uy, uz, (double *)f, (double *)h,
                                            (double *)prev, status);
    return cudaGetLastError();
}

cudaError_t launch_macro(int fp32, int N, long long ps, const void *f, const void *h, double *out,
                         unsigned *status, cudaStream_t s)
{
    const int b = 128, g = (N + b - 1) / b;
    if (fp32)
        macro_kernel<float><<<g, b, 0, s>>>(N, ps, (const float *)f, (const float *)h, out, status);
    else
        macro_kernel<double><<<g, b, 0, s>>>(N, ps, (const double *)f, (const double *)h, out,
                                             status);
    return cudaGetLastError();
}

int totals_blocks(int N)
{
    const int want = (N + kTotBlock - 1) / kTotBlock;
    return want < 1 ? 1 : (want > 1216 ? 1216 : want);   // 1216 = 8 x 152 SMs
}

cudaError_t launch_totals(int fp32, int N, long long ps, const void *f, const void *h,
                          double *partial, double *out, cudaStream_t s)
{
    const int nb = totals_blocks(N);
    if (fp32)
        totals_kernel<float><<<nb, kTotBlock, 0, s>>>(N, ps, (const float *)f, (const float *)h,
                                                      partial);
    else
        totals_kernel<double><<<nb, kTotBlock, 0, s>>>(N, ps, (const double *)f, (const double *)h,
                                                       partial);
    totals_finish<<<1, 32, 0, s>>>(nb, partial, out);
    return cudaGetLastError();
}

}  // namespace rlb
