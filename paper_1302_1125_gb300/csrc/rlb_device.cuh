// rlb_device.cuh -- per-cell physics of the ultra-relativistic lattice
// Boltzmann step (Mohseni, Mendoza, Succi, Herrmann, arXiv:1302.1125) as
// device functions: lattice constants, moments, Landau-frame recovery,
// equilibria, relaxation time, minmod streaming.
//
// Lattice units: delta x = 1, c = k_B = 1, nu = sqrt(13) so c_a = 1 and the
// lattice velocities are the integer vectors of Eq. 42 (LAT = 0); the basic
// D3Q19 lattice of Sec. II (LAT = 1) has nu = sqrt(19), c_a = 1 and unit
// diagonals.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "rlb_consts.h"

namespace rlb {

// integer velocity components c_i (c_a = 1; the diagonals carry 2 c_a)
struct Dir {
    int x, y, z;
};
constexpr Dir kDir[19] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                          {0, 0, 1},   {0, 0, -1},  {2, 2, 0},   {2, -2, 0},  {-2, 2, 0},
                          {-2, -2, 0}, {2, 0, 2},   {2, 0, -2},  {-2, 0, 2},  {-2, 0, -2},
                          {0, 2, 2},   {0, 2, -2},  {0, -2, 2},  {0, -2, -2}};

template <int I>
__host__ __device__ constexpr int shell()
{
    return I == 0 ? 0 : (I <= 6 ? 1 : 2);
}
// component A of c_i on lattice LAT (the basic lattice's diagonals are c_a,
// half the extended lattice's 2 c_a)
template <int I, int A, int LAT = 0>
__host__ __device__ constexpr int cdir()
{
    return (A == 0 ? kDir[I].x : (A == 1 ? kDir[I].y : kDir[I].z)) / (LAT == 1 && shell<I>() == 2 ? 2 : 1);
}

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_INLET = 2 };
enum { ST_NONPHYSICAL = 1, ST_ASYMMETRIC = 2, ST_TIMEOUT = 4 };   // ST_ASYMMETRIC: a state the 2-D symmetry
                                                                 // reduction cannot take; ST_TIMEOUT: a bounded
                                                                 // wait of a kernel gave up

// ---------------------------------------------------------------------------
// Macroscopic state and recovery (Sec. II: T^{0 mu} plus eps = 3P, Eq. 38)
// ---------------------------------------------------------------------------
struct Macro {
    double P, ux, uy, uz, n;   // u' = gamma u (spatial part of U^mu)
};

// Landau frame for eps = 3P: E = 4 P gamma^2 - P, M = 4 P gamma^2 u.  The
// eigenvalue is eps = 3 (E^2 - |M|^2) / (E + sqrt(4 E^2 - 3 |M|^2)); then
// gamma^2 = (E + P) / (4 P), u' = M / (4 P gamma), n = N^0 / gamma.
__host__ __device__ __forceinline__ bool recover(double E, double Mx, double My, double Mz, double N0,
                                        Macro &m)
{
    const double M2 = Mx * Mx + My * My + Mz * Mz;
    const double D = E * E - M2;
    const double eps = 3.0 * D / (E + sqrt(4.0 * E * E - 3.0 * M2));
    const double P = eps * (1.0 / 3.0);
    const double g2 = (E + P) / (4.0 * P);
    const double g = sqrt(g2);
    const double s = 1.0 / (4.0 * P * g);
    m.P = P;
    m.ux = Mx * s;
    m.uy = My * s;
    m.uz = Mz * s;
    m.n = N0 / g;
    return (E > 0.0) && (D > 0.0) && isfinite(m.n) && isfinite(s);
}

// tau from eta/s (Eq. 41 with s = n (4 - ln lambda), lambda = n / n_eq,
// n_eq = 16 T^3 / pi^2, T = P/n, Sec. III): tau = 1/2 + nu^2 (eta/s)(4 - ln lambda)/(4 T)
template <int LAT = 0>
__device__ __forceinline__ double tau_of(double P, double n, double eta_over_s)
{
    const double T = P / n;
    const double lam = n * kPi2Over16 / (T * T * T);
    const double sfac = fmax(4.0 - log(lam), kSMin);
    return 0.5 + Lat<LAT>::nu2 * eta_over_s * sfac / (4.0 * T);
}

// ---------------------------------------------------------------------------
// Equilibria as coefficient sets.  With integer c_i:
//   f_i^eq = w_i [K0 + sum_a c_a Kb_a + sum_a c_a^2 Kd_a + sum_{a<b} c_a c_b Ko_ab]
// is the second-order polynomial in u' whose lattice moments give
// T^{mu nu} = 4 P U^mu U^nu - P eta^{mu nu} (Eq. 36): with A = P / sigma2 =
// 13 P / 9, K0 = A (1 - 16/15 |u'|^2), Kb = A (4 gamma / xi0) u',
// Kd = A (52/15) u'^2, Ko = 13 A u'_a u'_b.
//   h_i^eq = w'_i n gamma (c0/ct + 3 c.u + 9/2 (c.u)^2 - 3/2 |u|^2)  (Eq. 58)
// gives H0 = B (c0/ct - 3/2 |u|^2), Hb = 3 B u, Hd = 9/2 B u^2,
// Ho = 9 B u_a u_b with B = n gamma.
// ---------------------------------------------------------------------------
template <typename R>
struct Coef {
    R K0, Kb[3], Kd[3], Ko[3];   // Ko order: xy, xz, yz
};

template <int LAT = 0>
__host__ __device__ __forceinline__ void coef_f(const Macro &m, Coef<double> &k)
{
    const double u2 = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    const double g = sqrt(1.0 + u2);
    const double A = m.P * Lat<LAT>::inv_sigma2;
    const double b = A * Lat<LAT>::four_over_xi0 * g;
    const double d = A * Lat<LAT>::a3f;
    const double o = A * Lat<LAT>::a2f;
    k.K0 = A * (1.0 - (16.0 / 15.0) * u2);
    k.Kb[0] = b * m.ux;
    k.Kb[1] = b * m.uy;
    k.Kb[2] = b * m.uz;
    k.Kd[0] = d * m.ux * m.ux;
    k.Kd[1] = d * m.uy * m.uy;
    k.Kd[2] = d * m.uz * m.uz;
    k.Ko[0] = o * m.ux * m.uy;
    k.Ko[1] = o * m.ux * m.uz;
    k.Ko[2] = o * m.uy * m.uz;
}

template <int LAT = 0>
__host__ __device__ __forceinline__ void coef_h(const Macro &m, Coef<double> &k)
{
    const double u2p = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    const double g = sqrt(1.0 + u2p);
    const double ig = 1.0 / g;
    const double ux = m.ux * ig, uy = m.uy * ig, uz = m.uz * ig;
    const double B = m.n * g;
    k.K0 = B * (Lat<LAT>::c0ct - 1.5 * (ux * ux + uy * uy + uz * uz));
    k.Kb[0] = 3.0 * B * ux;
    k.Kb[1] = 3.0 * B * uy;
    k.Kb[2] = 3.0 * B * uz;
    k.Kd[0] = 4.5 * B * ux * ux;
    k.Kd[1] = 4.5 * B * uy * uy;
    k.Kd[2] = 4.5 * B * uz * uz;
    k.Ko[0] = 9.0 * B * ux * uy;
    k.Ko[1] = 9.0 * B * ux * uz;
    k.Ko[2] = 9.0 * B * uy * uz;
}

// An equilibrium with the lattice weights and the diagonal factors (2 and 4
// on the extended lattice, 1 on the basic one) folded into its coefficients
// in double precision, so that a float form
// rounds each coefficient once instead of carrying a fixed rounding of the
// weights into every population (that fixed rounding would bias the moment
// sums, and so the conserved totals, the same way at every step).
template <typename R>
struct EqW {
    R r0;                          // rest:     w0 K0
    R a0, ab[3], ad[3];            // axis:     w1 K0, w1 Kb, w1 Kd
    R d0, db[3], dd[3], dk[3];     // diagonal: w2 K0, 2 w2 Kb, 4 w2 Kd, 4 w2 Ko
};

// DM = |c_ia| of a diagonal population (2 extended, 1 basic)
template <typename R, int DM = 2>
__host__ __device__ __forceinline__ EqW<R> weigh(const Coef<double> &k, double w0, double w1,
                                                 double w2)
{
    EqW<R> e;
    e.r0 = R(w0 * k.K0);
    e.a0 = R(w1 * k.K0);
    e.d0 = R(w2 * k.K0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        e.ab[j] = R(w1 * k.Kb[j]);
        e.ad[j] = R(w1 * k.Kd[j]);
        e.db[j] = R(double(DM) * w2 * k.Kb[j]);
        e.dd[j] = R(double(DM * DM) * w2 * k.Kd[j]);
        e.dk[j] = R(double(DM * DM) * w2 * k.Ko[j]);
    }
    return e;
}
template <typename R, int LAT = 0>
__host__ __device__ __forceinline__ EqW<R> weigh_f(const Coef<double> &k)
{
    return weigh<R, Lat<LAT>::dmag>(k, Lat<LAT>::w0, Lat<LAT>::w1, Lat<LAT>::w2);
}
template <typename R, int LAT = 0>
__host__ __device__ __forceinline__ EqW<R> weigh_h(const Coef<double> &k)
{
    return weigh<R, Lat<LAT>::dmag>(k, Lat<LAT>::wh0, Lat<LAT>::wh1, Lat<LAT>::wh2);
}

// 2 k(t) - k(t - dt), the extrapolated equilibrium of Eq. 57
__host__ __device__ __forceinline__ Coef<double> extrapolate(const Coef<double> &a,
                                                             const Coef<double> &b)
{
    Coef<double> k;
    k.K0 = 2.0 * a.K0 - b.K0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        k.Kb[j] = 2.0 * a.Kb[j] - b.Kb[j];
        k.Kd[j] = 2.0 * a.Kd[j] - b.Kd[j];
        k.Ko[j] = 2.0 * a.Ko[j] - b.Ko[j];
    }
    return k;
}

// population I of an equilibrium: f_i = w_i [K0 + sum_a c_a Kb_a +
// sum_a c_a^2 Kd_a + sum_{a<b} c_a c_b Ko_ab], with only the terms of the
// nonzero lattice components generated
template <int I, typename R>
__host__ __device__ __forceinline__ R eq_pop(const EqW<R> &e)
{
    constexpr int cx = cdir<I, 0>(), cy = cdir<I, 1>(), cz = cdir<I, 2>();
    constexpr int sh = shell<I>();
    if constexpr (sh == 0) {
        return e.r0;
    } else if constexpr (sh == 1) {
        constexpr int a = cx != 0 ? 0 : (cy != 0 ? 1 : 2);
        constexpr int s = cx + cy + cz;   // +1 or -1
        return s > 0 ? (e.a0 + e.ad[a]) + e.ab[a] : (e.a0 + e.ad[a]) - e.ab[a];
    } else {
        constexpr int a = cx != 0 ? 0 : 1;                 // first nonzero axis
        constexpr int b = cz != 0 ? 2 : 1;                 // second nonzero axis
        constexpr int ca = a == 0 ? cx : cy, cb = b == 2 ? cz : cy;
        constexpr int ko = (a == 0 && b == 1) ? 0 : ((a == 0 && b == 2) ? 1 : 2);
        R v = e.d0 + e.dd[a] + e.dd[b];
        v = (ca > 0) ? v + e.db[a] : v - e.db[a];
        v = (cb > 0) ? v + e.db[b] : v - e.db[b];
        v = (ca * cb > 0) ? v + e.dk[ko] : v - e.dk[ko];
        return v;
    }
}

// ---------------------------------------------------------------------------
// Streaming (Eqs. 47-53) and the minmod limiter
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R minmod(R a, R b)
{
    const R m = fmin(fabs(a), fabs(b));
    return (a > R(0) && b > R(0)) ? m : ((a < R(0) && b < R(0)) ? -m : R(0));
}

// Eq. 53 for doubles on the bit patterns, so that the limiter issues integer
// instructions instead of occupying the FP64 pipe (GB300: 2 per clock per
// SM): the magnitudes of non-negative doubles order as unsigned integers,
// the signs agree when the top bits do.  The value equals the floating-point
// form's (a zero may carry the sign of a).
template <>
__device__ __forceinline__ double minmod<double>(double a, double b)
{
    const unsigned long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    constexpr unsigned long long kSign = 0x8000000000000000ULL;
    const unsigned long long ma = ia & ~kSign, mb = ib & ~kSign;
    const unsigned long long m = ma < mb ? ma : mb;
    return __longlong_as_double(((ia ^ ib) & kSign) ? 0ULL : (m | (ia & kSign)));
}

// Neighbour map of one axis: linear offsets of the cells at d = -2, -1, +1, +2
// after the boundary rule, and a mask of inlet ghost cells.
struct AxisNbr {
    int off[4];
    unsigned ghost;
};

__device__ __forceinline__ AxisNbr axis_map(int c, int n, int stride, int lo, int hi)
{
    AxisNbr r;
    r.ghost = 0u;
    const int ds[4] = {-2, -1, 1, 2};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int cc = c + ds[k];
        if (cc < 0 || cc >= n) {
            const int bc = cc < 0 ? lo : hi;
            if (bc == BC_PERIODIC) {
                cc %= n;
                if (cc < 0) cc += n;
            } else if (bc == BC_OUTFLOW) {
                cc = cc < 0 ? 0 : n - 1;
            } else {
                r.ghost |= 1u << k;
                cc = c;
            }
        }
        r.off[k] = (cc - c) * stride;
    }
    return r;
}

}  // namespace rlb
