// rlb_cellops_f32.cuh -- initialisation and macroscopic output of the
// FP32-storage layout, two cells per thread in float and double-float
// arithmetic like the step kernel.  On GB300 the FP64 pipe issues 2
// operations per clock per SM against 128 float lanes, and the double
// forms of these per-cell operations (about 300 FP64 operations a cell)
// ran some twenty times longer than their loads and stores take.
#pragma once

#include "rlb_step_f32.cuh"

namespace rlb {
namespace f32 {

// Two cells: lane 0 reads source index s0 and writes destination index d0,
// lane 1 the same with s1, d1, written only when has1 (s1 = s0, d1 = d0
// otherwise).  VEC: d0 and s0 are even, d1 = d0 + 1 and s1 = s0 + 1, so a
// float plane of even stride moves the pair as one 8-byte access.
struct CellPair {
    long long s0, s1, d0, d1;
    bool has1;
};

template <bool VEC>
__device__ __forceinline__ void st_cells(float *q, const CellPair &c, f2 v)
{
    if (VEC && c.has1) {
        *reinterpret_cast<float2 *>(q + c.d0) = make_float2(v.x, v.y);
    } else {
        q[c.d0] = v.x;
        if (c.has1) q[c.d1] = v.y;
    }
}

template <bool VEC>
__device__ __forceinline__ f2 ld_cells(const float *q, const CellPair &c)
{
    if (VEC && c.has1) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(q + c.s0));
        return f2{v.x, v.y};
    }
    return f2{__ldg(q + c.s0), __ldg(q + c.s1)};
}

// c_a v for the integer lattice component c_a (|c_a| <= 2): exact
template <int C>
__device__ __forceinline__ f2 times_c(f2 v)
{
    static_assert(C >= -2 && C <= 2 && C != 0, "lattice component");
    if constexpr (C == 1) return v;
    else if constexpr (C == -1) return -v;
    else if constexpr (C == 2) return v + v;
    else return -(v + v);
}

// raw moment sums S = sum f, V_a = sum c_a f, Sh = sum h of the populations
// at the pair's destination planes (double-float accumulation)
template <int LAT>
struct RawSums {
    df2 S, Vx, Vy, Vz, H;
    __device__ __forceinline__ RawSums()
        : S{bc(0.0f), bc(0.0f)}, Vx{bc(0.0f), bc(0.0f)}, Vy{bc(0.0f), bc(0.0f)}, Vz{bc(0.0f), bc(0.0f)},
          H{bc(0.0f), bc(0.0f)} {}
    template <int I>
    __device__ __forceinline__ void add(f2 fv, f2 hv)
    {
        acc(S, fv);
        acc(H, hv);
        constexpr int cx = cdir<I, 0, LAT>(), cy = cdir<I, 1, LAT>(), cz = cdir<I, 2, LAT>();
        if constexpr (cx != 0) acc(Vx, times_c<cx>(fv));
        if constexpr (cy != 0) acc(Vy, times_c<cy>(fv));
        if constexpr (cz != 0) acc(Vz, times_c<cz>(fv));
    }
};

// weights folded into the coefficients, every population evaluated on its
// own (the rest one as w0 K0), so that each carries the roundings of its own
// terms only
template <int DM>
__device__ __forceinline__ W2 weigh2_direct(f2 K0, const f2 (&Kb)[3], const f2 (&Kd)[3], const f2 (&Ko)[3],
                                            float w0, float w1, float w2)
{
    W2 e;
    e.r0 = bc(w0) * K0;
    e.a0 = bc(w1) * K0;
    e.d0 = bc(w2) * K0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        e.ab[j] = bc(w1) * Kb[j];
        e.ad[j] = bc(w1) * Kd[j];
        e.db[j] = bc(float(DM) * w2) * Kb[j];
        e.dd[j] = bc(float(DM * DM) * w2) * Kd[j];
        e.dk[j] = bc(float(DM * DM) * w2) * Ko[j];
    }
    return e;
}

// f = f^eq(P = n T, u), h = h^eq(n, u) (Eqs. 43-45 and 46) for the input
// cells s0, s1 (n, T, velocity v; uy, uz may be NULL for zero), stored at
// plane indices d0, d1; the previous level is the raw sums of the stored
// populations.  Validity and 1 - |v|^2 are taken in double, the rest in
// float.
template <int LAT, bool VEC>
__device__ __forceinline__ void init_pair(const CellPair &c, long long ps, const double *__restrict__ n,
                                          const double *__restrict__ Tt, const double *__restrict__ ux,
                                          const double *__restrict__ uy, const double *__restrict__ uz,
                                          float *__restrict__ f, float *__restrict__ h,
                                          float *__restrict__ prev, unsigned *status)
{
    float Pv[2], nv[2], vv[3][2], om[2];
    const long long src[2] = {c.s0, c.s1};
    bool ok = true;
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const long long i = src[l];
        const double a = ux[i], b = uy ? uy[i] : 0.0, d = uz ? uz[i] : 0.0;
        const double one_m = 1.0 - (a * a + b * b + d * d);
        const double nd = n[i], Td = Tt[i];
        Pv[l] = float(nd * Td);
        nv[l] = float(nd);
        om[l] = float(one_m);
        vv[0][l] = float(a);
        vv[1][l] = float(b);
        vv[2][l] = float(d);
        ok = ok && nd > 0.0 && Td > 0.0 && nv[l] > 0.0f && Pv[l] > 0.0f && isfinite(Pv[l]) && om[l] > 0.0f;
    }
    if (!ok) atomicOr(status, unsigned(ST_NONPHYSICAL));
    const f2 g = f2{1.0f / sqrtf(om[0]), 1.0f / sqrtf(om[1])};
    Mac2 m;
    m.P = f2{Pv[0], Pv[1]};
    m.n = f2{nv[0], nv[1]};
    m.ux = g * f2{vv[0][0], vv[0][1]};
    m.uy = g * f2{vv[1][0], vv[1][1]};
    m.uz = g * f2{vv[2][0], vv[2][1]};

    f2 K0, Kb[3], Kd[3], Ko[3];
    coef_f2<LAT>(m, K0, Kb, Kd, Ko);
    const W2 ef = weigh2_direct<Lat<LAT>::dmag>(K0, Kb, Kd, Ko, float(Lat<LAT>::w0), float(Lat<LAT>::w1),
                                                float(Lat<LAT>::w2));
    coef_h2<LAT>(m, K0, Kb, Kd, Ko);
    const W2 eh = weigh2_direct<Lat<LAT>::dmag>(K0, Kb, Kd, Ko, float(Lat<LAT>::wh0), float(Lat<LAT>::wh1),
                                                float(Lat<LAT>::wh2));
    RawSums<LAT> r;
    for_pops(RLB_F32_POPS, [&](auto ic) {
        constexpr int I = decltype(ic)::value;
        const f2 fv = eq2<I>(ef), hv = eq2<I>(eh);
        st_cells<VEC>(f + I * ps, c, fv);
        st_cells<VEC>(h + I * ps, c, hv);
        r.template add<I>(fv, hv);
    });
    st_cells<VEC>(prev + 0 * ps, c, r.S.hi + r.S.lo);
    st_cells<VEC>(prev + 1 * ps, c, r.Vx.hi + r.Vx.lo);
    st_cells<VEC>(prev + 2 * ps, c, r.Vy.hi + r.Vy.lo);
    st_cells<VEC>(prev + 3 * ps, c, r.Vz.hi + r.Vz.lo);
    st_cells<VEC>(prev + 4 * ps, c, r.H.hi + r.H.lo);
}

// moments and Landau-frame recovery (Eq. 36, the eigenvalue problem of
// Sec. II.B) of the populations at plane indices s0, s1: n, e = 3P, v_x,
// v_y, v_z, gamma written to out[k * ostride + d]
template <int LAT, bool VEC>
__device__ __forceinline__ void macro_pair(const CellPair &c, long long ps, const float *__restrict__ f,
                                           const float *__restrict__ h, double *__restrict__ out,
                                           long long ostride, unsigned *status)
{
    RawSums<LAT> r;
    for_pops(RLB_F32_POPS, [&](auto ic) {
        constexpr int I = decltype(ic)::value;
        r.template add<I>(ld_cells<VEC>(f + I * ps, c), ld_cells<VEC>(h + I * ps, c));
    });
    bool ok0, ok1;
    const Mac2 m = recover2<LAT, false>(r.S, r.Vx, r.Vy, r.Vz, r.H.hi + r.H.lo, ok0, ok1);
    if (!ok0 || (c.has1 && !ok1)) atomicOr(status, unsigned(ST_NONPHYSICAL));
    const f2 u2 = fma2(m.ux, m.ux, fma2(m.uy, m.uy, m.uz * m.uz));
    const f2 g = f2{sqrtf(1.0f + u2.x), sqrtf(1.0f + u2.y)};
    const f2 vals[6] = {m.n, bc(3.0f) * m.P, f2{m.ux.x / g.x, m.ux.y / g.y}, f2{m.uy.x / g.x, m.uy.y / g.y},
                        f2{m.uz.x / g.x, m.uz.y / g.y}, g};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        out[k * ostride + c.d0] = double(vals[k].x);
        if (c.has1) out[k * ostride + c.d1] = double(vals[k].y);
    }
}

}  // namespace f32
}  // namespace rlb
