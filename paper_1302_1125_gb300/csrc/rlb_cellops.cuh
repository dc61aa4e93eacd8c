// rlb_cellops.cuh -- per-cell initialisation and macroscopic output of the FP64
// form (the FP32-storage form has its own, in float arithmetic:
// rlb_cellops_f32.cuh).
#pragma once

#include "rlb_kernels.cuh"

namespace rlb {

// f = f^eq(P = nT, u), h = h^eq(n, u), previous level = this state, for the
// input cell `in` stored at plane index `idx`
template <typename T, int LAT = 0>
__device__ __forceinline__ void init_cell(long long in, long long idx, long long ps, const double *__restrict__ n,
                                          const double *__restrict__ Tt, const double *__restrict__ ux,
                                          const double *__restrict__ uy, const double *__restrict__ uz,
                                          T *__restrict__ f, T *__restrict__ h, T *__restrict__ prev,
                                          unsigned *status)
{
    const double vx = ux[in], vy = uy ? uy[in] : 0.0, vz = uz ? uz[in] : 0.0;
    const double v2 = vx * vx + vy * vy + vz * vz;
    const double g = 1.0 / sqrt(1.0 - v2);
    if (!(n[in] > 0.0 && Tt[in] > 0.0 && v2 < 1.0 && isfinite(n[in] * Tt[in]) && isfinite(g)))
        atomicOr(status, unsigned(ST_NONPHYSICAL));
    Macro m;
    m.P = n[in] * Tt[in];
    m.ux = g * vx;
    m.uy = g * vy;
    m.uz = g * vz;
    m.n = n[in];
    Coef<double> a;
    coef_f<LAT>(m, a);
    const EqW<T> kf = weigh_f<T, LAT>(a);
    coef_h<LAT>(m, a);
    const EqW<T> kh = weigh_h<T, LAT>(a);
    for_pops(RLB_POPS, [&](auto ic) {
        constexpr int I = decltype(ic)::value;
        f[I * ps + idx] = eq_pop<I>(kf);
        h[I * ps + idx] = eq_pop<I>(kh);
    });
    prev[0 * ps + idx] = T(m.P);
    prev[1 * ps + idx] = T(m.ux);
    prev[2 * ps + idx] = T(m.uy);
    prev[3 * ps + idx] = T(m.uz);
    prev[4 * ps + idx] = T(m.n);
}

// moments + recovery of the populations at plane index `idx`: n, e, u_x,
// u_y, u_z, gamma written to out[k * ostride + o]
template <typename T, int LAT = 0>
__device__ __forceinline__ void macro_cell(long long idx, long long ps, const T *__restrict__ f,
                                           const T *__restrict__ h, double *__restrict__ out, long long o,
                                           long long ostride, unsigned *status)
{
    double sf = 0.0, sh = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    for_pops(RLB_POPS, [&](auto ic) {
        constexpr int I = decltype(ic)::value;
        const double fv = double(f[I * ps + idx]);
        sf += fv;
        sh += double(h[I * ps + idx]);
        if constexpr (cdir<I, 0, LAT>() != 0) mx += double(cdir<I, 0, LAT>()) * fv;
        if constexpr (cdir<I, 1, LAT>() != 0) my += double(cdir<I, 1, LAT>()) * fv;
        if constexpr (cdir<I, 2, LAT>() != 0) mz += double(cdir<I, 2, LAT>()) * fv;
    });
    Macro m;
    if (!recover(Lat<LAT>::xi0sq * sf, Lat<LAT>::xi0 * mx, Lat<LAT>::xi0 * my, Lat<LAT>::xi0 * mz,
                 Lat<LAT>::xi0 * sh, m))
        atomicOr(status, unsigned(ST_NONPHYSICAL));
    const double g = sqrt(1.0 + m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
    out[0 * ostride + o] = m.n;
    out[1 * ostride + o] = 3.0 * m.P;
    out[2 * ostride + o] = m.ux / g;
    out[3 * ostride + o] = m.uy / g;
    out[4 * ostride + o] = m.uz / g;
    out[5 * ostride + o] = g;
}

}  // namespace rlb
