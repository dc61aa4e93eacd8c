// rlb_kernels.cuh -- kernels of the fused RLB time step.
//
// One thread updates one cell: it reads the 19 + 19 local populations,
// forms the moments and the Landau-frame macroscopic state of time t,
// evaluates the extrapolated equilibria 2 f^eq(t) - f^eq(t - dt) from the
// current and the stored previous macroscopic state, streams every
// population with the minmod flux difference of its own neighbours
// (plus the bulk Laplacian for f), applies the implicit update of Eq. 57
// and writes the populations of t + dt and the macroscopic state of t.
#pragma once

#include <utility>

#include "rlb_classes.cuh"
#include "rlb_device.cuh"
#include "rlb_internal.h"

namespace rlb {

template <int... Is, typename F>
__device__ __forceinline__ void for_pops(std::integer_sequence<int, Is...>, F &&fn)
{
    (fn(std::integral_constant<int, Is>{}), ...);
}
#define RLB_POPS std::make_integer_sequence<int, 19>{}

template <typename T>
__device__ __forceinline__ T ldg(const T *p)
{
    return __ldg(p);
}

// value of a neighbour (slot k of the axis map) or the inlet ghost value
template <typename T>
__device__ __forceinline__ T nbr(const T *q, int idx, const AxisNbr &a, int k, T ghost)
{
    return ((a.ghost >> k) & 1u) ? ghost : ldg(q + idx + a.off[k]);
}

// Streaming terms of one population along axis A (Eqs. 47-53): the
// accumulator acc receives minus dt (c0/ct) times the conservative minmod
// flux difference h^a(x) - h^a(x - e_a); for f with i != 0 the neighbour sum
// s receives q(x + e_A) + q(x - e_A) of the bulk term's second difference
// (assigned on the first axis, FIRST).
template <typename T, bool IS_F, int I, int A, int LAT, bool FIRST>
__device__ __forceinline__ void axis_terms(const T *q, int idx, const AxisNbr &an, T qc, T ghost,
                                           T k1, T k2, T hl, T &acc, T &s)
{
    constexpr int c = cdir<I, A, LAT>();
    constexpr bool need_lap = IS_F && I != 0;
    auto add_s = [&](T qm1, T qp1) {
        if constexpr (need_lap) {
            if constexpr (FIRST) s = qp1 + qm1;
            else s += qp1 + qm1;
        }
    };
    if constexpr (c > 0) {
        const T qm2 = nbr(q, idx, an, 0, ghost);
        const T qm1 = nbr(q, idx, an, 1, ghost);
        const T qp1 = nbr(q, idx, an, 2, ghost);
        const T d0 = qm1 - qm2, d1 = qc - qm1, d2 = qp1 - qc;
        const T D = d1 + hl * (minmod(d2, d1) - minmod(d1, d0));
        acc -= (c == 1 ? k1 : k2) * D;
        add_s(qm1, qp1);
    } else if constexpr (c < 0) {
        const T qm1 = nbr(q, idx, an, 1, ghost);
        const T qp1 = nbr(q, idx, an, 2, ghost);
        const T qp2 = nbr(q, idx, an, 3, ghost);
        const T e0 = qc - qm1, e1 = qp1 - qc, e2 = qp2 - qp1;
        const T D = e1 - hl * (minmod(e1, e2) - minmod(e0, e1));
        acc += (c == -1 ? k1 : k2) * D;
        add_s(qm1, qp1);
    } else if constexpr (need_lap) {
        add_s(nbr(q, idx, an, 1, ghost), nbr(q, idx, an, 2, ghost));
    }
}

// f + streaming (+ bulk) for population I: the explicit part of Eq. 57.  The
// bulk term's central second difference sum_A [q(x + e_A) - 2 q(x) + q(x - e_A)]
// is taken as s - 2 DIM q(x) in one fused operation (exact coefficients, so
// that its sum over a periodic grid carries no systematic rounding).
template <typename T, int DIM, bool IS_F, int I, int LAT>
__device__ __forceinline__ T streamed(const T *q, int idx, const AxisNbr (&am)[3], T qc, T ghost,
                                      T k1, T k2, T hl, T kbulk)
{
    constexpr bool need_lap = IS_F && I != 0;
    T acc = qc, s = T(0);
    axis_terms<T, IS_F, I, 0, LAT, true>(q, idx, am[0], qc, ghost, k1, k2, hl, acc, s);
    if constexpr (DIM > 1) axis_terms<T, IS_F, I, 1, LAT, false>(q, idx, am[1], qc, ghost, k1, k2, hl, acc, s);
    if constexpr (DIM > 2) axis_terms<T, IS_F, I, 2, LAT, false>(q, idx, am[2], qc, ghost, k1, k2, hl, acc, s);
    if constexpr (need_lap) acc += kbulk * fma(T(-2 * DIM), qc, s);
    return acc;
}

template <typename T>
__device__ __forceinline__ void flag(const StepParams &p, unsigned bits)
{
    atomicOr(p.status, bits);
}

// LIN: blocks of one row of threads take consecutive cells of the x-fastest
// order (grids whose nx, ny do not fill the tiles); otherwise blocks of
// 32 x 4 threads take tiles of 32 x 4 cells in one z-plane (the 1-D form:
// one row of tiles)
// NP = 7 or 14: the 1-D or 2-D symmetry reduction (rlb_classes.cuh); only
// the class representatives' planes are read and written
template <typename T, int DIM, bool EULER, int LAT, bool LIN = false, int NP = 19>
__global__ void __launch_bounds__(128) step_kernel(const StepParams p, const T *__restrict__ f,
                                                   const T *__restrict__ h, T *__restrict__ fo,
                                                   T *__restrict__ ho, T *__restrict__ prev)
{
    int x, y, z;
    if constexpr (LIN) {
        const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
        const unsigned row = t / unsigned(p.nx);
        x = int(t - row * unsigned(p.nx));
        y = int(row % unsigned(p.ny));
        z = int(row / unsigned(p.ny));
        if (z >= p.nz) return;
    } else {
        x = blockIdx.x * blockDim.x + threadIdx.x;
        y = blockIdx.y * blockDim.y + threadIdx.y;
        z = blockIdx.z;
        if (x >= p.nx || y >= p.ny) return;
    }
    const int idx = x + p.nx * (y + p.ny * z);
    const long long ps = p.ps;

    AxisNbr am[3];
    am[0] = axis_map(x, p.nx, 1, p.bc_lo[0], p.bc_hi[0]);
    if (DIM > 1) am[1] = axis_map(y, p.ny, p.nx, p.bc_lo[1], p.bc_hi[1]);
    if (DIM > 2) am[2] = axis_map(z, p.nz, p.nx * p.ny, p.bc_lo[2], p.bc_hi[2]);

    const T k1 = T(p.k1), k2 = T(p.k2), hl = T(p.half_lim), kbulk = T(p.kbulk);

    static_assert(NP == 19 || (NP == 7 && DIM == 1 && !EULER) || (NP == 14 && DIM == 2 && !EULER),
                  "the symmetry reductions are 1-D or 2-D and viscous");
    if constexpr (!EULER) {
        // moments of f(t), h(t) at the cell (Eq. 36 with p_i^0 = xi0); class k
        // counts mult(k) equal populations (powers of two: exact scaling)
        T fl[NP], hq[NP];
        double sf = 0.0, sh = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
        for_pops(std::make_integer_sequence<int, NP>{}, [&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int I = rep<NP>(k), m = mult<NP>(k);
            fl[k] = ldg(f + I * ps + idx);
            hq[k] = ldg(h + I * ps + idx);
            const double fv = double(fl[k]);
            sf += m == 1 ? fv : double(m) * fv;
            sh += m == 1 ? double(hq[k]) : double(m) * double(hq[k]);
            if constexpr (cdir<I, 0, LAT>() != 0) mx += double(cdir<I, 0, LAT>() * m) * fv;
            if constexpr (has_vy<NP>() && cdir<I, 1, LAT>() != 0) my += double(cdir<I, 1, LAT>() * m) * fv;
            if constexpr (has_vz<NP>() && cdir<I, 2, LAT>() != 0) mz += double(cdir<I, 2, LAT>() * m) * fv;
        });
        Macro mt;
        const bool ok = recover(Lat<LAT>::xi0sq * sf, Lat<LAT>::xi0 * mx, Lat<LAT>::xi0 * my, Lat<LAT>::xi0 * mz, Lat<LAT>::xi0 * sh, mt);
        if (!ok) flag<T>(p, ST_NONPHYSICAL);
        const double tau = p.tau_override > 0.0 ? p.tau_override : tau_of<LAT>(mt.P, mt.n, p.eta_over_s);
        const double omega = p.kw / tau;
        // f(t+dt) = pre + kappa (G - pre), kappa = omega / (1 + omega): Eq. 57
        // solved for f(t+dt), in the form whose rounding does not scale the
        // conserved sums
        const T kap = T(omega / (1.0 + omega));

        Macro mp;
        mp.P = double(prev[0 * ps + idx]);
        mp.ux = double(prev[1 * ps + idx]);
        mp.uy = double(prev[2 * ps + idx]);
        mp.uz = double(prev[3 * ps + idx]);
        mp.n = double(prev[4 * ps + idx]);
        Coef<double> a, b;
        coef_f<LAT>(mt, a);
        coef_f<LAT>(mp, b);
        const EqW<T> kf = weigh_f<T, LAT>(extrapolate(a, b));
        coef_h<LAT>(mt, a);
        coef_h<LAT>(mp, b);
        const EqW<T> kh = weigh_h<T, LAT>(extrapolate(a, b));

        for_pops(std::make_integer_sequence<int, NP>{}, [&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int I = rep<NP>(k);
            const T pre = streamed<T, DIM, true, I, LAT>(f + I * ps, idx, am, fl[k], T(p.ghost_f[I]), k1,
                                                    k2, hl, kbulk);
            fo[I * ps + idx] = pre + kap * (eq_pop<I>(kf) - pre);
        });
        for_pops(std::make_integer_sequence<int, NP>{}, [&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int I = rep<NP>(k);
            const T pre = streamed<T, DIM, false, I, LAT>(h + I * ps, idx, am, hq[k], T(p.ghost_h[I]),
                                                     k1, k2, hl, kbulk);
            ho[I * ps + idx] = pre + kap * (eq_pop<I>(kh) - pre);
        });
        prev[0 * ps + idx] = T(mt.P);
        prev[1 * ps + idx] = T(mt.ux);
        prev[2 * ps + idx] = T(mt.uy);
        prev[3 * ps + idx] = T(mt.uz);
        prev[4 * ps + idx] = T(mt.n);
    } else {
        // Euler mode (Sec. III): f, h <- equilibria of the streamed state
        double sf = 0.0, sh = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
        for_pops(RLB_POPS, [&](auto ic) {
            constexpr int I = decltype(ic)::value;
            const T qc = ldg(f + I * ps + idx);
            const double fv = double(streamed<T, DIM, true, I, LAT>(f + I * ps, idx, am, qc,
                                                               T(p.ghost_f[I]), k1, k2, hl, kbulk));
            sf += fv;
            if constexpr (cdir<I, 0, LAT>() != 0) mx += double(cdir<I, 0, LAT>()) * fv;
            if constexpr (cdir<I, 1, LAT>() != 0) my += double(cdir<I, 1, LAT>()) * fv;
            if constexpr (cdir<I, 2, LAT>() != 0) mz += double(cdir<I, 2, LAT>()) * fv;
            const T qh = ldg(h + I * ps + idx);
            sh += double(streamed<T, DIM, false, I, LAT>(h + I * ps, idx, am, qh, T(p.ghost_h[I]), k1, k2,
                                                    hl, kbulk));
        });
        Macro mt;
        const bool ok = recover(Lat<LAT>::xi0sq * sf, Lat<LAT>::xi0 * mx, Lat<LAT>::xi0 * my, Lat<LAT>::xi0 * mz, Lat<LAT>::xi0 * sh, mt);
        if (!ok) flag<T>(p, ST_NONPHYSICAL);
        Coef<double> a;
        coef_f<LAT>(mt, a);
        const EqW<T> kf = weigh_f<T, LAT>(a);
        coef_h<LAT>(mt, a);
        const EqW<T> kh = weigh_h<T, LAT>(a);
        for_pops(RLB_POPS, [&](auto ic) {
            constexpr int I = decltype(ic)::value;
            fo[I * ps + idx] = eq_pop<I>(kf);
            ho[I * ps + idx] = eq_pop<I>(kh);
        });
        prev[0 * ps + idx] = T(mt.P);
        prev[1 * ps + idx] = T(mt.ux);
        prev[2 * ps + idx] = T(mt.uy);
        prev[3 * ps + idx] = T(mt.uz);
        prev[4 * ps + idx] = T(mt.n);
    }
}

}  // namespace rlb
