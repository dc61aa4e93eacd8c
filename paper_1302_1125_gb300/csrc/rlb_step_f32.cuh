// rlb_step_f32.cuh -- the fused step of the FP32-storage form.
//
// One thread updates two x-adjacent cells (x0, x0 + 1) of one (y, z) row.
// Populations are stored, streamed and relaxed in FP32.  The moment sums
// T^00 and T^0a are accumulated error-free as double-float pairs (TwoSum),
// and E^2 - |M|^2, the quantity whose cancellation grows like gamma^2 in the
// Landau-frame recovery, is formed in double-float before one rounding; the
// rest of the recovery (a well-conditioned function of E^2 - |M|^2, E, M and
// N^0), tau and the equilibrium coefficients are FP32.  No FP64 instruction
// is issued.  The previous level's recovery is the same arithmetic on its
// stored float sums.  The REC64 variant (rlb_options.recovery_fp64) runs
// both recoveries in FP64 from the exact double values of the sums instead;
// it exists to measure what FP64 buys over the double-float form.
//
// Conservation: the float equilibrium coefficients carry fixed roundings of
// irrational constants (weights, 4/xi0, 13/9, ...) that would bias their
// lattice moments identically at every step.  The previous level is kept as
// the raw moment sums of time t - dt (sum f, sum c_a f, sum h), so the
// moments 2 f^eq(t) - f^eq(t - dt) must have are known exactly; after the
// coefficients are formed, their closed-form lattice sums are compared with
// those targets and the rest coefficient (T^00, N^0) and the axis
// first-order coefficient (T^0a) absorb the difference, so only unbiased
// per-cell roundings remain.
#pragma once

#include <utility>

#include "rlb_bulk.cuh"
#include "rlb_classes.cuh"
#include "rlb_device.cuh"
#include "rlb_internal.h"
#include "rlb_pair.cuh"

namespace rlb {

namespace f32 {

// xi0^2 split into float hi + lo where a double-float value is needed
template <int LAT>
struct Xi0Sq {
    static constexpr float hi = float(Lat<LAT>::xi0sq);
    static constexpr float lo = float(Lat<LAT>::xi0sq - double(float(Lat<LAT>::xi0sq)));
};

template <int... Is, typename F>
__device__ __forceinline__ void for_pops(std::integer_sequence<int, Is...>, F &&fn)
{
    (fn(std::integral_constant<int, Is>{}), ...);
}
#define RLB_F32_POPS std::make_integer_sequence<int, 19>{}

// the population classes of the symmetry reductions (rlb_classes.cuh)
using rlb::has_vy;
using rlb::has_vz;
using rlb::mult;
using rlb::rep;

// geometry of one thread's pair of cells
struct Geo {
    int idx0, idx1;      // cell indices (idx1 = idx0 when x0 + 1 is outside the grid)
    int x0;
    bool has1;
    int oa, oc;          // offsets of the pairs holding x0-2, x0-1 and x0+2, x0+3
    unsigned xfix;       // edge columns: clamp or ghost fix-ups (XF_*)
    int yoff[4], zoff[4];   // offsets of rows/planes at -2, -1, +1, +2 (mapped)
    // 3-D staged step: byte offsets, from the start of a population plane, of
    // the pairs a thread stages: x0-2, x0, x0+2 (mapped like oa, oc), then the
    // rows at y-2, y-1, y+1, y+2 and the planes at z-2 .. z+2 (mapped); 32
    // bits hold them since FP32 grids have fewer than 2^30 cells
    unsigned sb[11];
};
// XF_HI_ODD1 / XF_HI_ODD3: odd-length tube stored with one pad cell, the pair
// holds its last cell (x0 = nx - 1) or ends two cells before it (x0 = nx - 3)
enum { XF_LO_CLAMP = 1, XF_LO_GHOST = 2, XF_HI_CLAMP = 4, XF_HI_GHOST = 8, XF_HI_ODD1 = 16, XF_HI_ODD3 = 32 };

__device__ __forceinline__ int map1(int c, int n, int lo, int hi, bool &ghost)
{
    ghost = false;
    if (c >= 0 && c < n) return c;
    const int bc = c < 0 ? lo : hi;
    if (bc == BC_PERIODIC) {
        int m = c % n;
        return m < 0 ? m + n : m;
    }
    if (bc == BC_OUTFLOW) return c < 0 ? 0 : n - 1;
    ghost = true;
    return c < 0 ? 0 : n - 1;
}

// Load kinds.  LD_NC: read-only path, for a launch that never writes the
// populations it reads.  A persistent launch reads what it wrote in earlier
// steps: LD_CA (cached in L1) when only threads of the same block wrote the
// data (ordered by the block barrier), LD_CG (cached in L2 only) when other
// blocks of the cluster wrote it on other SMs.
enum { LD_NC = 0, LD_CA = 1, LD_CG = 2 };
template <int LD>
__device__ __forceinline__ f2 ld2(const float *q)
{
    const float2 *p = reinterpret_cast<const float2 *>(q);
    float2 v;
    if constexpr (LD == LD_CG) v = __ldcg(p);
    else if constexpr (LD == LD_CA) v = __ldca(p);
    else v = __ldg(p);
    return f2{v.x, v.y};
}
template <int LD>
__device__ __forceinline__ float ld1(const float *q)
{
    if constexpr (LD == LD_CG) return __ldcg(q);
    else if constexpr (LD == LD_CA) return __ldca(q);
    else return __ldg(q);
}

// the pair of cells (x0, x0+1) at element offset `off` from idx0
template <bool VEC2, int LD = LD_NC>
__device__ __forceinline__ f2 ldpair(const float *q, const Geo &g, int off)
{
    if constexpr (VEC2) return ld2<LD>(q + g.idx0 + off);
    else return f2{ld1<LD>(q + g.idx0 + off), ld1<LD>(q + g.idx1 + off)};
}

template <bool VEC2>
__device__ __forceinline__ void stpair(float *q, const Geo &g, f2 v)
{
    if constexpr (VEC2) {
        *reinterpret_cast<float2 *>(q + g.idx0) = make_float2(v.x, v.y);
    } else {
        q[g.idx0] = v.x;
        if (g.has1) q[g.idx1] = v.y;
    }
}

// one value of the x-stencil through the boundary map (odd nx only)
static __device__ __noinline__ float xval_mapped(const float *q, int idx0, int x0, int k, const StepParams &p,
                                          float ghost)
{
    bool gh;
    const int c = map1(x0 - 2 + k, p.nx, p.bc_lo[0], p.bc_hi[0], gh);
    return gh ? ghost : __ldg(q + idx0 + (c - x0));
}

// Where the stencil values of one population come from: straight from global
// memory (GlobalSrc), or from this thread's shared-memory staging slots that
// asynchronous copies filled earlier (StageSrc).  get(slot, off) returns the
// pair at element offset `off` from idx0; `slot` is its staging slot: 0, 1, 2
// for x0-2, x0, x0+2, then 3 + 3 (A - 1) + k for the k-th neighbour pair along
// axis A (see stage_item).
template <bool VEC2, int LD>
struct GlobalSrc {
    const float *q;
    const Geo &g;
    __device__ __forceinline__ f2 get(int, int off) const { return ldpair<VEC2, LD>(q, g, off); }
    template <int A, int D>
    __device__ __forceinline__ f2 nb(int slot, int off) const { return get(slot, off); }
};

struct StageSrc {
    const f2 *s;     // slot 0 of this thread's buffer
    int stride;      // f2 elements between slots
    __device__ __forceinline__ f2 get(int slot, int) const { return s[slot * stride]; }
    template <int A, int D>
    __device__ __forceinline__ f2 nb(int slot, int off) const { return get(slot, off); }
};
// TileSrc (rlb_bulk.cuh): the block's bulk-copied tiles; it takes the
// neighbours along y and z by axis and distance, the x pairs by slot

// x0-2 .. x0+3 of one plane.  With even nx every thread loads three aligned
// pairs; periodic edges wrap to aligned pairs, and the clamped (open) or ghost
// (inlet) positions of the two edge columns are patched afterwards.
template <bool VEC2, int LD, typename Src>
__device__ __forceinline__ void xstencil(const Src &src, const float *q, const Geo &g, const StepParams &p,
                                         float ghost, float (&v)[6])
{
    if constexpr (VEC2) {
        const f2 a = src.get(0, g.oa), b = src.get(1, 0), c = src.get(2, g.oc);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
        if (g.xfix) {
            if (g.xfix & XF_LO_CLAMP) { v[0] = v[2]; v[1] = v[2]; }
            if (g.xfix & XF_LO_GHOST) { v[0] = ghost; v[1] = ghost; }
            if (g.xfix & XF_HI_CLAMP) { v[4] = v[3]; v[5] = v[3]; }
            if (g.xfix & XF_HI_GHOST) { v[4] = ghost; v[5] = ghost; }
            if (g.xfix & XF_HI_ODD1) { v[3] = v[2]; v[4] = v[2]; v[5] = v[2]; }
            if (g.xfix & XF_HI_ODD3) v[5] = v[4];
        }
    } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = xval_mapped(q, g.idx0, g.x0, k, p, ghost);
    }
}

// element offset of the row (A = 1) or plane (A = 2) at distance d
template <int A>
__device__ __forceinline__ int off_of(const Geo &g, const StepParams &p, int d)
{
    const int k = d < 0 ? d + 2 : d + 1;
    if constexpr (A == 1) return g.yoff[k];
    else return g.zoff[k];
}

// Divisions and the logarithm of the per-cell scalar work (recovery, tau,
// kappa, 1/gamma): the fast intrinsics (a few ulp, operands far from the
// range limits of __fdividef) unless RLB_F32_IEEE_DIV is defined.  The
// conserved sums do not depend on them: the equilibrium's lattice sums are
// set to exact targets afterwards (weigh2).
__device__ __forceinline__ float fdiv(float a, float b)
{
#ifdef RLB_F32_IEEE_DIV
    return a / b;
#else
    return __fdividef(a, b);
#endif
}
__device__ __forceinline__ float flog(float a)
{
#ifdef RLB_F32_IEEE_DIV
    return logf(a);
#else
    return __logf(a);
#endif
}

struct Mac2 {
    f2 P, ux, uy, uz, n;
};

// equilibrium coefficients of a pair, weights and diagonal factors folded in
struct W2 {
    f2 r0, a0, ab[3], ad[3], d0, db[3], dd[3], dk[3];
};

// K0, Kb, Kd, Ko of the f equilibrium (see rlb_device.cuh) for a pair
template <int LAT>
__device__ __forceinline__ void coef_f2(const Mac2 &m, f2 &K0, f2 (&Kb)[3], f2 (&Kd)[3], f2 (&Ko)[3])
{
    const f2 u2 = fma2(m.ux, m.ux, fma2(m.uy, m.uy, m.uz * m.uz));
    const f2 g = f2{sqrtf(1.0f + u2.x), sqrtf(1.0f + u2.y)};
    const f2 A = m.P * bc(Lat<LAT>::f_inv_sigma2);
    K0 = A * fma2(bc(-16.0f / 15.0f), u2, bc(1.0f));
    const f2 b = A * bc(float(Lat<LAT>::four_over_xi0)) * g;
    Kb[0] = b * m.ux; Kb[1] = b * m.uy; Kb[2] = b * m.uz;
    const f2 d = A * bc(Lat<LAT>::f_a3f);
    Kd[0] = d * m.ux * m.ux; Kd[1] = d * m.uy * m.uy; Kd[2] = d * m.uz * m.uz;
    const f2 o = A * bc(Lat<LAT>::f_a2f);
    Ko[0] = o * m.ux * m.uy; Ko[1] = o * m.ux * m.uz; Ko[2] = o * m.uy * m.uz;
}

template <int LAT>
__device__ __forceinline__ void coef_h2(const Mac2 &m, f2 &K0, f2 (&Kb)[3], f2 (&Kd)[3], f2 (&Ko)[3])
{
    const f2 u2p = fma2(m.ux, m.ux, fma2(m.uy, m.uy, m.uz * m.uz));
    const f2 g = f2{sqrtf(1.0f + u2p.x), sqrtf(1.0f + u2p.y)};
    const f2 ig = f2{fdiv(1.0f, g.x), fdiv(1.0f, g.y)};
    const f2 ux = m.ux * ig, uy = m.uy * ig, uz = m.uz * ig;
    const f2 B = m.n * g;
    const f2 uu = fma2(ux, ux, fma2(uy, uy, uz * uz));
    K0 = B * fma2(bc(-1.5f), uu, bc(float(Lat<LAT>::c0ct)));
    const f2 b3 = B * bc(3.0f);
    Kb[0] = b3 * ux; Kb[1] = b3 * uy; Kb[2] = b3 * uz;
    const f2 b45 = B * bc(4.5f);
    Kd[0] = b45 * ux * ux; Kd[1] = b45 * uy * uy; Kd[2] = b45 * uz * uz;
    const f2 b9 = B * bc(9.0f);
    Ko[0] = b9 * ux * uy; Ko[1] = b9 * ux * uz; Ko[2] = b9 * uy * uz;
}

// weights folded in (Eqs. 43-45 or 59-60) and the lattice sums set to the
// exact targets: T0 = sum_i G_i, Ta = sum_i c_ia G_i (only for f).  The rest
// weight w0 enters only through the target (sum_i w_i = 1).
template <int DM>
__device__ __forceinline__ W2 weigh2(f2 K0, const f2 (&Kb)[3], const f2 (&Kd)[3], const f2 (&Ko)[3],
                                     float w0, float w1, float w2, f2 T0, const f2 *Ta)
{
    (void)w0;
    W2 e;
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
    // sum_i G_i = r0 + 6 a0 + 12 d0 + 2 sum ad + 8 sum dd: the rest coefficient
    // is the remainder that makes this equal T0, with the other terms summed
    // error-free (their roundings are correlated, all being K0 times fixed
    // weights, and a float sum of them is biased); one final rounding
    df2 R{bc(0.0f), bc(0.0f)};
    {
        const f2 p6 = bc(6.0f) * e.a0, p12 = bc(12.0f) * e.d0;
        acc(R, p6);
        acc(R, fma2(bc(6.0f), e.a0, -p6));
        acc(R, p12);
        acc(R, fma2(bc(12.0f), e.d0, -p12));
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        acc(R, e.ad[j] + e.ad[j]);
        acc(R, bc(8.0f) * e.dd[j]);
    }
    {
        f2 s, er;
        two_sum(T0, -R.hi, s, er);
        e.r0 = s + (er - R.lo);
    }
    if (Ta) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            // sum_i c_ia G_i = 2 ab_a + 8 DM db_a (8 DM db and the halving are exact)
            e.ab[j] = bc(0.5f) * (Ta[j] - bc(float(8 * DM)) * e.db[j]);
        }
    }
    return e;
}

template <int I>
__device__ __forceinline__ f2 eq2(const W2 &e)
{
    constexpr int cx = cdir<I, 0>(), cy = cdir<I, 1>(), cz = cdir<I, 2>();
    constexpr int sh = shell<I>();
    if constexpr (sh == 0) {
        return e.r0;
    } else if constexpr (sh == 1) {
        constexpr int a = cx != 0 ? 0 : (cy != 0 ? 1 : 2);
        constexpr int s = cx + cy + cz;
        const f2 base = e.a0 + e.ad[a];
        return s > 0 ? base + e.ab[a] : base - e.ab[a];
    } else {
        constexpr int a = cx != 0 ? 0 : 1;
        constexpr int b = cz != 0 ? 2 : 1;
        constexpr int ca = a == 0 ? cx : cy, cb = b == 2 ? cz : cy;
        constexpr int ko = (a == 0 && b == 1) ? 0 : ((a == 0 && b == 2) ? 1 : 2);
        f2 v = e.d0 + (e.dd[a] + e.dd[b]);
        v = ca > 0 ? v + e.db[a] : v - e.db[a];
        v = cb > 0 ? v + e.db[b] : v - e.db[b];
        v = ca * cb > 0 ? v + e.dk[ko] : v - e.dk[ko];
        return v;
    }
}

// Landau-frame recovery of a pair from the raw sums S = sum f, V_a = sum c_a f
// (double-float) and Sh = sum h: E = xi0^2 S, M = xi0 V,
// E^2 - |M|^2 = xi0^2 (xi0^2 S^2 - |V|^2) formed in double-float,
// P = (E^2 - |M|^2) / (E + sqrt(E^2 + 3 (E^2 - |M|^2))), gamma^2 = (E + P)/(4 P),
// u' = M / (4 P gamma), n = N^0 / gamma
// (FAST = false: IEEE division, for the macroscopic output)
template <int LAT, bool FAST = true>
__device__ __forceinline__ Mac2 recover2(const df2 &S, const df2 &Vx, const df2 &Vy, const df2 &Vz,
                                         f2 Sh, bool &ok0, bool &ok1)
{
    constexpr float kXi0 = float(Lat<LAT>::xi0), kXi0Sq = float(Lat<LAT>::xi0sq);
    auto dv = [](float a, float b) {
        if constexpr (FAST) return fdiv(a, b);
        else return a / b;
    };
    const df2 V2 = dadd(dadd(sq(Vx), sq(Vy)), sq(Vz));
    const df2 Dr = dadd(dscale(sq(S), Xi0Sq<LAT>::hi, Xi0Sq<LAT>::lo), dneg(V2));
    const f2 D = bc(kXi0Sq) * (Dr.hi + Dr.lo);
    const f2 E = bc(kXi0Sq) * (S.hi + S.lo);
    const f2 root2 = fma2(E, E, bc(3.0f) * D);
    const f2 den = E + f2{sqrtf(root2.x), sqrtf(root2.y)};
    Mac2 m;
    m.P = f2{dv(D.x, den.x), dv(D.y, den.y)};
    const f2 fourP = bc(4.0f) * m.P;
    const f2 g2 = f2{dv(E.x + m.P.x, fourP.x), dv(E.y + m.P.y, fourP.y)};
    const f2 g = f2{sqrtf(g2.x), sqrtf(g2.y)};
    const f2 s = f2{dv(kXi0, fourP.x * g.x), dv(kXi0, fourP.y * g.y)};
    m.ux = (Vx.hi + Vx.lo) * s;
    m.uy = (Vy.hi + Vy.lo) * s;
    m.uz = (Vz.hi + Vz.lo) * s;
    m.n = f2{dv(kXi0 * Sh.x, g.x), dv(kXi0 * Sh.y, g.y)};
    ok0 = E.x > 0.0f && D.x > 0.0f && isfinite(m.n.x) && isfinite(s.x);
    ok1 = E.y > 0.0f && D.y > 0.0f && isfinite(m.n.y) && isfinite(s.y);
    return m;
}

// The same recovery in FP64 (REC64 step variant): the double-float sums are
// converted to double exactly (hi + lo), the Landau-frame recovery runs in
// double arithmetic (rlb_device.cuh: recover, IEEE division and square root)
// and its results are rounded once to float for the equilibrium coefficients.
template <int LAT>
__device__ __forceinline__ Mac2 recover2_64(const df2 &S, const df2 &Vx, const df2 &Vy, const df2 &Vz,
                                            const df2 &Hs, bool &ok0, bool &ok1)
{
    constexpr double xi0 = Lat<LAT>::xi0, xi0sq = Lat<LAT>::xi0sq;
    auto dd = [](float hi, float lo) { return double(hi) + double(lo); };
    Macro a, b;
    ok0 = recover(xi0sq * dd(S.hi.x, S.lo.x), xi0 * dd(Vx.hi.x, Vx.lo.x), xi0 * dd(Vy.hi.x, Vy.lo.x),
                  xi0 * dd(Vz.hi.x, Vz.lo.x), xi0 * dd(Hs.hi.x, Hs.lo.x), a);
    ok1 = recover(xi0sq * dd(S.hi.y, S.lo.y), xi0 * dd(Vx.hi.y, Vx.lo.y), xi0 * dd(Vy.hi.y, Vy.lo.y),
                  xi0 * dd(Vz.hi.y, Vz.lo.y), xi0 * dd(Hs.hi.y, Hs.lo.y), b);
    Mac2 m;
    m.P = f2{float(a.P), float(b.P)};
    m.ux = f2{float(a.ux), float(b.ux)};
    m.uy = f2{float(a.uy), float(b.uy)};
    m.uz = f2{float(a.uz), float(b.uz)};
    m.n = f2{float(a.n), float(b.n)};
    return m;
}

// a float sum as a double-float with zero low part
__device__ __forceinline__ df2 as_df2(f2 v) { return df2{v, bc(0.0f)}; }

// tau from eta/s (Eq. 41 with the entropy of Sec. III), float
template <int LAT>
__device__ __forceinline__ float tau1(float P, float n, float eta_over_s)
{
    const float T = fdiv(P, n);
    const float lam = fdiv(n * float(kPi2Over16), T * T * T);
    const float sfac = fmaxf(4.0f - flog(lam), float(kSMin));
    return 0.5f + fdiv(Lat<LAT>::f_nu2 * eta_over_s * sfac, 4.0f * T);
}

// streaming increment of population I along axis A for the pair (+ bulk lap)
template <bool IS_F, int I, int A, int LAT, typename Src>
__device__ __forceinline__ void axis2(const Src &src, const Geo &g, const StepParams &p, const float (&xv)[6],
                                      f2 C, float k1, float k2, float hl, f2 &inc, f2 &lap)
{
    constexpr int sb = 3 * A;   // first staging slot of axis A (A = 1, 2)
    constexpr int c = cdir<I, A, LAT>();
    constexpr bool need_lap = IS_F && I != 0;
    const float k = (c == 1 || c == -1) ? k1 : k2;
    if constexpr (A == 0) {
        if constexpr (c > 0) {
            const float dm3 = xv[1] - xv[0], dm1 = xv[2] - xv[1], dp1 = xv[3] - xv[2], dp3 = xv[4] - xv[3];
            const float mA = mm(dp1, dm1), mB = mm(dm1, dm3), mC = mm(dp3, dp1);
            const f2 D = fma2(bc(hl), mk(mA, mC) - mk(mB, mA), mk(dm1, dp1));
            inc = fma2(bc(-k), D, inc);
            if constexpr (need_lap) lap = lap + (mk(dp1, dp3) - mk(dm1, dp1));
        } else if constexpr (c < 0) {
            const float dm1 = xv[2] - xv[1], dp1 = xv[3] - xv[2], dp3 = xv[4] - xv[3], dp5 = xv[5] - xv[4];
            const float m1 = mm(dm1, dp1), m2 = mm(dp1, dp3), m3 = mm(dp3, dp5);
            const f2 D = fma2(bc(-hl), mk(m2, m3) - mk(m1, m2), mk(dp1, dp3));
            inc = fma2(bc(k), D, inc);
            if constexpr (need_lap) lap = lap + (mk(dp1, dp3) - mk(dm1, dp1));
        } else if constexpr (need_lap) {
            const float dm1 = xv[2] - xv[1], dp1 = xv[3] - xv[2], dp3 = xv[4] - xv[3];
            lap = lap + (mk(dp1, dp3) - mk(dm1, dp1));
        }
    } else {
        if constexpr (c > 0) {
            const f2 Aq = src.template nb<A, -2>(sb, off_of<A>(g, p, -2));
            const f2 B = src.template nb<A, -1>(sb + 1, off_of<A>(g, p, -1));
            const f2 Dq = src.template nb<A, 1>(sb + 2, off_of<A>(g, p, 1));
            const f2 d0 = B - Aq, d1 = C - B, d2 = Dq - C;
            const f2 Dv = fma2(bc(hl), mm(d2, d1) - mm(d1, d0), d1);
            inc = fma2(bc(-k), Dv, inc);
            if constexpr (need_lap) lap = lap + (d2 - d1);
        } else if constexpr (c < 0) {
            const f2 B = src.template nb<A, -1>(sb, off_of<A>(g, p, -1));
            const f2 Dq = src.template nb<A, 1>(sb + 1, off_of<A>(g, p, 1));
            const f2 Eq = src.template nb<A, 2>(sb + 2, off_of<A>(g, p, 2));
            const f2 e0 = C - B, e1 = Dq - C, e2 = Eq - Dq;
            const f2 Dv = fma2(bc(-hl), mm(e1, e2) - mm(e0, e1), e1);
            inc = fma2(bc(k), Dv, inc);
            if constexpr (need_lap) lap = lap + (e1 - e0);
        } else if constexpr (need_lap) {
            const f2 B = src.template nb<A, -1>(sb, off_of<A>(g, p, -1));
            const f2 Dq = src.template nb<A, 1>(sb + 1, off_of<A>(g, p, 1));
            lap = lap + ((Dq - C) - (C - B));
        }
    }
}

// f (or h) + streaming (+ bulk) of population I for the pair: the explicit part of Eq. 57
template <int DIM, bool IS_F, int I, bool VEC2, int LD, int LAT, typename Src>
__device__ __forceinline__ f2 streamed2(const Src &src, const float *q, const Geo &g, const StepParams &p,
                                        float ghost, float k1, float k2, float hl, float kb)
{
    constexpr bool xneed = cdir<I, 0, LAT>() != 0 || (IS_F && I != 0);
    float xv[6];
    f2 C;
    if constexpr (xneed) {
        xstencil<VEC2, LD>(src, q, g, p, ghost, xv);
        C = mk(xv[2], xv[3]);
    } else {
        C = src.get(1, 0);
    }
    f2 inc = bc(0.0f), lap = bc(0.0f);
    if constexpr (xneed) axis2<IS_F, I, 0, LAT>(src, g, p, xv, C, k1, k2, hl, inc, lap);
    if constexpr (DIM > 1) axis2<IS_F, I, 1, LAT>(src, g, p, xv, C, k1, k2, hl, inc, lap);
    if constexpr (DIM > 2) axis2<IS_F, I, 2, LAT>(src, g, p, xv, C, k1, k2, hl, inc, lap);
    if constexpr (IS_F && I != 0) inc = fma2(bc(kb), lap, inc);
    return C + inc;
}

// Asynchronous copies (cp.async, cached in L1) into shared memory, completed
// per thread by cp.async.wait_group: no other thread reads the slots.
__device__ __forceinline__ void cp8(unsigned dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

#ifndef RLB_STAGE_BUFS
#define RLB_STAGE_BUFS 3
#endif
// pairs staged per population: 3 along x, 3 along each other streamed axis
template <int DIM>
constexpr int stage_slots()
{
    return 3 * DIM;
}
constexpr int kStageBufs = RLB_STAGE_BUFS;   // populations in flight: the one computed and the next ones
constexpr int kStageAhead = kStageBufs - 1;  // prefetch distance in populations

// Issue the copies of item J (J < NP: f class J, else h class J - NP) into
// staging buffer J % kStageBufs: the same pairs, in the same
// slots, that streamed2 reads through StageSrc.  dst0 = shared address of
// slot 0 of buffer 0 of this thread, sstride = bytes between slots.
template <int DIM, int NP, int J, int LAT>
__device__ __forceinline__ void stage_item(const float *f, const float *h, const Geo &g, const StepParams &p,
                                           long long ps, unsigned dst0, unsigned sstride)
{
    constexpr bool IS_F = J < NP;
    constexpr int I = rep<NP>(IS_F ? J : J - NP);
    constexpr bool xneed = cdir<I, 0, LAT>() != 0 || (IS_F && I != 0);
    constexpr bool need_lap = IS_F && I != 0;
    const unsigned d = dst0 + unsigned(J % kStageBufs) * stage_slots<DIM>() * sstride;
    if constexpr (DIM == 3) {
        // one population plane base for the block, the thread's fixed byte
        // offsets on top (fewer address instructions than a per-thread base)
        const char *qb = reinterpret_cast<const char *>((IS_F ? f : h) + I * ps);
        auto at = [&](int s) { return reinterpret_cast<const float *>(qb + g.sb[s]); };
        if constexpr (xneed) {
            cp8(d + 0 * sstride, at(0));
            cp8(d + 2 * sstride, at(2));
        }
        cp8(d + 1 * sstride, at(1));
        auto axis = [&](auto ac) {
            constexpr int A = decltype(ac)::value;
            constexpr int c = cdir<I, A, LAT>();
            constexpr int s0 = 3 + 4 * (A - 1);   // slots of distances -2, -1, +1, +2
            const unsigned b = d + unsigned(3 * A) * sstride;
            if constexpr (c > 0) {
                cp8(b, at(s0 + 0));
                cp8(b + sstride, at(s0 + 1));
                cp8(b + 2 * sstride, at(s0 + 2));
            } else if constexpr (c < 0) {
                cp8(b, at(s0 + 1));
                cp8(b + sstride, at(s0 + 2));
                cp8(b + 2 * sstride, at(s0 + 3));
            } else if constexpr (need_lap) {
                cp8(b, at(s0 + 1));
                cp8(b + sstride, at(s0 + 2));
            }
        };
        axis(std::integral_constant<int, 1>{});
        axis(std::integral_constant<int, 2>{});
        cp_commit();
        return;
    }
    const float *q = (IS_F ? f : h) + I * ps + g.idx0;
    if constexpr (xneed) {
        cp8(d + 0 * sstride, q + g.oa);
        cp8(d + 2 * sstride, q + g.oc);
    }
    cp8(d + 1 * sstride, q);
    auto axis = [&](auto ac) {
        constexpr int A = decltype(ac)::value;
        constexpr int c = cdir<I, A, LAT>();
        const unsigned b = d + unsigned(3 * A) * sstride;
        if constexpr (c > 0) {
            cp8(b, q + off_of<A>(g, p, -2));
            cp8(b + sstride, q + off_of<A>(g, p, -1));
            cp8(b + 2 * sstride, q + off_of<A>(g, p, 1));
        } else if constexpr (c < 0) {
            cp8(b, q + off_of<A>(g, p, -1));
            cp8(b + sstride, q + off_of<A>(g, p, 1));
            cp8(b + 2 * sstride, q + off_of<A>(g, p, 2));
        } else if constexpr (need_lap) {
            cp8(b, q + off_of<A>(g, p, -1));
            cp8(b + sstride, q + off_of<A>(g, p, 1));
        }
    };
    if constexpr (DIM > 1) axis(std::integral_constant<int, 1>{});
    if constexpr (DIM > 2) axis(std::integral_constant<int, 2>{});
    cp_commit();
}

// The update of one pair of cells (Eq. 57 for f and h), shared by the grid
// kernel and the batched tube kernel.  eos = eta/s and kb = the bulk
// prefactor of the cell's grid or tube.
//
// park (PARK = true): this thread's slots in shared memory, slot k at
// park[k * pstride]; the h-equilibrium coefficients wait there while the f
// populations are updated, which frees their registers for the f loop.
//
// stage (STAGE = true, even nx, viscous step): the stencil of each population
// is copied asynchronously into this thread's shared-memory slots
// kStageAhead populations ahead of its use (stage_item), so that the loads of the next
// populations are in flight while one is computed; stage = slot 0 of buffer
// 0 of this thread, sstride = f2 elements between slots.
//
// NP = 7 or 14: the 1-D or 2-D symmetry reduction (see rep and mult); only
// the planes of the class representatives are read and written, and the
// previous level's planes of the zero sums (sum c_z f; 1-D also sum c_y f)
// are left alone.
template <int DIM, bool EULER, bool VEC2, int LD = LD_NC, bool PARK = false, bool STAGE = false, int NP = 19,
          int LAT = 0, bool REC64 = false, bool BULK = false>
__device__ __forceinline__ void update_pair(const StepParams &p, const Geo &g, float eos, float kb,
                                            const float *__restrict__ f, const float *__restrict__ h,
                                            float *__restrict__ fo, float *__restrict__ ho,
                                            float *__restrict__ prev, long long ps,
                                            f2 *park = nullptr, int pstride = 0,
                                            f2 *stage = nullptr, int sstride = 0, Bulk *bk = nullptr)
{
    const float k1 = p.f_k1, k2 = p.f_k2, hl = p.f_half_lim;
    static_assert(!STAGE || (VEC2 && !EULER), "staging needs aligned pairs and the viscous step");
    static_assert(NP == 19 || (NP == 7 && DIM == 1 && !EULER) || (NP == 14 && DIM == 2 && !EULER),
                  "the symmetry reductions are 1-D or 2-D and viscous");
    static_assert(!REC64 || (!EULER && NP == 19), "the FP64 recovery is a variant of the viscous 19-population step");
    static_assert(!BULK || (DIM == 3 && VEC2 && !EULER && NP == 19 && !STAGE),
                  "bulk-copied tiles: the viscous 3-D step with aligned pairs");
    constexpr int NI = 2 * NP;   // items: f classes, then h classes
    unsigned sdst0 = 0;
    if constexpr (STAGE) {
        sdst0 = unsigned(__cvta_generic_to_shared(stage));
        for_pops(std::make_integer_sequence<int, kStageAhead>{}, [&](auto jc) {
            stage_item<DIM, NP, decltype(jc)::value, LAT>(f, h, g, p, ps, sdst0, unsigned(sstride * sizeof(f2)));
        });
    }
    // the explicit part of item J (J < NP: f class J, else h class J - NP)
    auto item = [&](auto jc) -> f2 {
        constexpr int J = decltype(jc)::value;
        constexpr bool IS_F = J < NP;
        constexpr int I = rep<NP>(IS_F ? J : J - NP);
        const float *q = (IS_F ? f : h) + I * ps;
        const float ghost = IS_F ? p.f_ghost_f[I] : p.f_ghost_h[I];
        if constexpr (BULK) {
            constexpr int b = J % kBulkBufs;
            constexpr unsigned par = unsigned(J / kBulkBufs) & 1u;
            if (!bk->failed && !mbar_wait(&bk->full[b], par)) {
                bk->failed = true;
                atomicOr(p.status, unsigned(ST_TIMEOUT));
            }
            bk->failed = __any_sync(0xffffffffu, bk->failed);   // warp-uniform: the issue below is warp-wide
            const TileSrc src{bk->ctr + b * kTileFloats, bk->zpl + b * kTileFloats};
            const f2 r = streamed2<DIM, IS_F, I, VEC2, LD, LAT>(src, q, g, p, ghost, k1, k2, hl, kb);
            // this warp is done with buffer b: it counts itself out, and the
            // warp that counts the last of the 8 refills the buffer with item
            // J + kBulkBufs (release fence before the count, acquire after
            // it, then the generic-to-async proxy fence before the copies
            // overwrite what the other warps read)
            if constexpr (J + kBulkBufs < NI) {
                __syncwarp();
                int last = 0;
                if (bk->lane == 0) {
                    asm volatile("fence.acq_rel.cta;" ::: "memory");
                    last = (atomicAdd(&bk->done[b], 1) & 7) == 7;
                    if (last) asm volatile("fence.acq_rel.cta;" ::: "memory");
                }
                if (__shfl_sync(0xffffffffu, last, 0) && !bk->failed) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bulk_issue<NP, J + kBulkBufs, LAT>(*bk, p, f, h);
                }
            }
            return r;
        } else if constexpr (STAGE) {
            if constexpr (J + kStageAhead < NI) {
                stage_item<DIM, NP, J + kStageAhead, LAT>(f, h, g, p, ps, sdst0, unsigned(sstride * sizeof(f2)));
                cp_wait<kStageAhead>();
            } else {
                cp_wait<NI - 1 - J>();   // the groups issued after item J's
            }
            const StageSrc src{stage + (J % kStageBufs) * stage_slots<DIM>() * sstride, sstride};
            return streamed2<DIM, IS_F, I, VEC2, LD, LAT>(src, q, g, p, ghost, k1, k2, hl, kb);
        } else {
            const GlobalSrc<VEC2, LD> src{q, g};
            return streamed2<DIM, IS_F, I, VEC2, LD, LAT>(src, q, g, p, ghost, k1, k2, hl, kb);
        }
    };

    if constexpr (!EULER) {
        // raw sums of the local populations: S = sum f, V_a = sum c_a f
        // (double-float), Sh = sum h
        df2 S{bc(0.0f), bc(0.0f)}, Vx = S, Vy = S, Vz = S, Hs = S;
        for_pops(std::make_integer_sequence<int, NP>{}, [&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int I = rep<NP>(k), m = mult<NP>(k);
            const f2 v = ldpair<VEC2, LD>(f + I * ps, g, 0);
            // m c_i v with m and c_i powers of two: exact
            auto scaled = [&](auto wc) {
                constexpr int w = decltype(wc)::value;
                return w == 1 ? v : (w == -1 ? -v : bc(float(w)) * v);
            };
            acc(S, scaled(std::integral_constant<int, m>{}));
            constexpr int cx = cdir<I, 0, LAT>(), cy = cdir<I, 1, LAT>(), cz = cdir<I, 2, LAT>();
            if constexpr (cx != 0) acc(Vx, scaled(std::integral_constant<int, cx * m>{}));
            // under a reduction sum c_y f (1-D) and sum c_z f are zero
            if constexpr (has_vy<NP>() && cy != 0) acc(Vy, scaled(std::integral_constant<int, cy * m>{}));
            if constexpr (has_vz<NP>() && cz != 0) acc(Vz, scaled(std::integral_constant<int, cz * m>{}));
            const f2 hv = ldpair<VEC2, LD>(h + I * ps, g, 0);
            acc(Hs, m == 1 ? hv : bc(float(m)) * hv);
        });
        const f2 Sh = Hs.hi + Hs.lo;
        bool ok0, ok1;
        Mac2 mt;
        if constexpr (REC64) mt = recover2_64<LAT>(S, Vx, Vy, Vz, Hs, ok0, ok1);
        else mt = recover2<LAT>(S, Vx, Vy, Vz, Sh, ok0, ok1);
        if (!ok0 || (g.has1 && !ok1)) atomicOr(p.status, unsigned(ST_NONPHYSICAL));

        f2 kap;
        {
            float t0, t1;
            if (p.f_tau_override > 0.0f) {
                t0 = t1 = p.f_tau_override;
            } else {
                t0 = tau1<LAT>(mt.P.x, mt.n.x, eos);
                t1 = tau1<LAT>(mt.P.y, mt.n.y, eos);
            }
            const float kw = p.f_kw;
            const float w0 = fdiv(kw, t0), w1 = fdiv(kw, t1);
            kap = f2{fdiv(w0, 1.0f + w0), fdiv(w1, 1.0f + w1)};
        }

        // the previous level holds the raw moment sums of time t - dt, so the
        // targets of 2 f^eq(t) - f^eq(t - dt) are exact: T = 2 S(t) - S(t - dt)
        const f2 Sp = ldpair<VEC2, LD>(prev + 0 * ps, g, 0);
        const f2 Vpx = ldpair<VEC2, LD>(prev + 1 * ps, g, 0);
        const f2 Vpy = has_vy<NP>() ? ldpair<VEC2, LD>(prev + 2 * ps, g, 0) : bc(0.0f);
        const f2 Vpz = has_vz<NP>() ? ldpair<VEC2, LD>(prev + 3 * ps, g, 0) : bc(0.0f);
        const f2 Shp = ldpair<VEC2, LD>(prev + 4 * ps, g, 0);
        // the previous level's recovery: the same arithmetic as this level's,
        // from its stored float sums.  Its validity is not checked again: the
        // same sums passed the check as the current level one step earlier
        // (or in rlb_init), and the flags' registers cost spills here.
        Mac2 mp;
        {
            bool okp0, okp1;
            if constexpr (REC64)
                mp = recover2_64<LAT>(as_df2(Sp), as_df2(Vpx), as_df2(Vpy), as_df2(Vpz), as_df2(Shp), okp0, okp1);
            else
                mp = recover2<LAT>(as_df2(Sp), as_df2(Vpx), as_df2(Vpy), as_df2(Vpz), Shp, okp0, okp1);
            (void)okp0;
            (void)okp1;
        }
        const f2 T0 = fma2(bc(2.0f), S.hi + S.lo, -Sp);
        f2 Ta[3];
        Ta[0] = fma2(bc(2.0f), Vx.hi + Vx.lo, -Vpx);
        Ta[1] = fma2(bc(2.0f), Vy.hi + Vy.lo, -Vpy);
        Ta[2] = fma2(bc(2.0f), Vz.hi + Vz.lo, -Vpz);

        // h coefficients of 2 h^eq(t) - h^eq(t - dt) (Eq. 58) and their N^0
        // target, formed now so that mt and mp die before the f loop
        f2 H0, Hb[3], Hd[3], Ho[3];
        {
            f2 L0, Lb[3], Ld[3], Lo[3];
            coef_h2<LAT>(mt, H0, Hb, Hd, Ho);
            coef_h2<LAT>(mp, L0, Lb, Ld, Lo);
            H0 = fma2(bc(2.0f), H0, -L0);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                Hb[j] = fma2(bc(2.0f), Hb[j], -Lb[j]);
                Hd[j] = fma2(bc(2.0f), Hd[j], -Ld[j]);
                Ho[j] = fma2(bc(2.0f), Ho[j], -Lo[j]);
            }
        }
        f2 T0h = fma2(bc(2.0f), Sh, -Shp);
        {
            f2 K0, Kb[3], Kd[3], Ko[3], L0, Lb[3], Ld[3], Lo[3];
            coef_f2<LAT>(mt, K0, Kb, Kd, Ko);
            coef_f2<LAT>(mp, L0, Lb, Ld, Lo);
            K0 = fma2(bc(2.0f), K0, -L0);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                Kb[j] = fma2(bc(2.0f), Kb[j], -Lb[j]);
                Kd[j] = fma2(bc(2.0f), Kd[j], -Ld[j]);
                Ko[j] = fma2(bc(2.0f), Ko[j], -Lo[j]);
            }
            const W2 ef = weigh2<Lat<LAT>::dmag>(K0, Kb, Kd, Ko, float(Lat<LAT>::w0), float(Lat<LAT>::w1), float(Lat<LAT>::w2), T0, Ta);
            // the raw sums of this level become the next step's previous level
            stpair<VEC2>(prev + 0 * ps, g, S.hi + S.lo);
            stpair<VEC2>(prev + 1 * ps, g, Vx.hi + Vx.lo);
            if constexpr (has_vy<NP>()) stpair<VEC2>(prev + 2 * ps, g, Vy.hi + Vy.lo);
            if constexpr (has_vz<NP>()) stpair<VEC2>(prev + 3 * ps, g, Vz.hi + Vz.lo);
            stpair<VEC2>(prev + 4 * ps, g, Sh);
            if constexpr (PARK) {
                park[0] = H0;
                park[10 * pstride] = T0h;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    park[(1 + j) * pstride] = Hb[j];
                    park[(4 + j) * pstride] = Hd[j];
                    park[(7 + j) * pstride] = Ho[j];
                }
            }
            for_pops(std::make_integer_sequence<int, NP>{}, [&](auto kc) {
                constexpr int k = decltype(kc)::value;
                constexpr int I = rep<NP>(k);
                const f2 pre = item(std::integral_constant<int, k>{});
                stpair<VEC2>(fo + I * ps, g, fma2(kap, eq2<I>(ef) - pre, pre));
            });
        }
        {
            if constexpr (PARK) {
                H0 = park[0];
                T0h = park[10 * pstride];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    Hb[j] = park[(1 + j) * pstride];
                    Hd[j] = park[(4 + j) * pstride];
                    Ho[j] = park[(7 + j) * pstride];
                }
            }
            const W2 eh = weigh2<Lat<LAT>::dmag>(H0, Hb, Hd, Ho, float(Lat<LAT>::wh0), float(Lat<LAT>::wh1), float(Lat<LAT>::wh2), T0h, nullptr);
            for_pops(std::make_integer_sequence<int, NP>{}, [&](auto kc) {
                constexpr int k = decltype(kc)::value;
                constexpr int I = rep<NP>(k);
                const f2 pre = item(std::integral_constant<int, NP + k>{});
                stpair<VEC2>(ho + I * ps, g, fma2(kap, eq2<I>(eh) - pre, pre));
            });
        }
    } else {
        // Euler mode (Sec. III): f, h <- equilibria of the streamed state
        df2 S{bc(0.0f), bc(0.0f)}, Vx = S, Vy = S, Vz = S, Hs = S;
        for_pops(RLB_F32_POPS, [&](auto ic) {
            constexpr int I = decltype(ic)::value;
            const f2 v = item(std::integral_constant<int, I>{});
            acc(S, v);
            constexpr int cx = cdir<I, 0, LAT>(), cy = cdir<I, 1, LAT>(), cz = cdir<I, 2, LAT>();
            if constexpr (cx != 0) acc(Vx, cx > 0 ? (cx == 1 ? v : v + v) : (cx == -1 ? -v : -(v + v)));
            if constexpr (cy != 0) acc(Vy, cy > 0 ? (cy == 1 ? v : v + v) : (cy == -1 ? -v : -(v + v)));
            if constexpr (cz != 0) acc(Vz, cz > 0 ? (cz == 1 ? v : v + v) : (cz == -1 ? -v : -(v + v)));
            acc(Hs, item(std::integral_constant<int, 19 + I>{}));
        });
        const f2 Sh = Hs.hi + Hs.lo;
        bool ok0, ok1;
        const Mac2 mt = recover2<LAT>(S, Vx, Vy, Vz, Sh, ok0, ok1);
        if (!ok0 || (g.has1 && !ok1)) atomicOr(p.status, unsigned(ST_NONPHYSICAL));
        const f2 Ta[3] = {Vx.hi + Vx.lo, Vy.hi + Vy.lo, Vz.hi + Vz.lo};
        f2 K0, Kb[3], Kd[3], Ko[3];
        coef_f2<LAT>(mt, K0, Kb, Kd, Ko);
        const W2 ef = weigh2<Lat<LAT>::dmag>(K0, Kb, Kd, Ko, float(Lat<LAT>::w0), float(Lat<LAT>::w1), float(Lat<LAT>::w2), S.hi + S.lo, Ta);
        coef_h2<LAT>(mt, K0, Kb, Kd, Ko);
        const W2 eh = weigh2<Lat<LAT>::dmag>(K0, Kb, Kd, Ko, float(Lat<LAT>::wh0), float(Lat<LAT>::wh1), float(Lat<LAT>::wh2), Sh, nullptr);
        for_pops(RLB_F32_POPS, [&](auto ic) {
            constexpr int I = decltype(ic)::value;
            stpair<VEC2>(fo + I * ps, g, eq2<I>(ef));
            stpair<VEC2>(ho + I * ps, g, eq2<I>(eh));
        });
        stpair<VEC2>(prev + 0 * ps, g, S.hi + S.lo);
        stpair<VEC2>(prev + 1 * ps, g, Ta[0]);
        stpair<VEC2>(prev + 2 * ps, g, Ta[1]);
        stpair<VEC2>(prev + 3 * ps, g, Ta[2]);
        stpair<VEC2>(prev + 4 * ps, g, Sh);
    }
}

// The tile (bx, by, bz) of this block when blocks are taken in slabs of
// slab_by block rows, z-planes in order within a slab (blocks start in the
// order of their linear index): the planes the z-stencils of the resident
// blocks read stay in L2 until the blocks of the neighbouring planes have
// read them, instead of a whole z-plane of the grid per step in z.
// slab_by = 0 or >= the block rows: the plain x, y, z order.
__device__ __forceinline__ void slab_order(int slab_by, unsigned &bx, unsigned &by, unsigned &bz)
{
    const unsigned nbx = gridDim.x, nby = gridDim.y, nbz = gridDim.z, sb = unsigned(slab_by);
    if (sb == 0u || sb >= nby) return;
    const unsigned L = blockIdx.x + nbx * (blockIdx.y + nby * blockIdx.z);
    const unsigned s = L / (nbx * sb * nbz);
    const unsigned rows = min(sb, nby - s * sb);
    const unsigned r = L - s * (nbx * sb * nbz);
    bz = r / (nbx * rows);
    const unsigned q = r - bz * (nbx * rows);
    by = s * sb + q / nbx;
    bx = q - (q / nbx) * nbx;
}

#ifndef RLB_F32_MINB
#define RLB_F32_MINB 2
#endif
#ifndef RLB_F32_BY
#define RLB_F32_BY 8
#endif

constexpr int kParkSlots = 11;   // f2 slots per thread in shared memory
#ifdef RLB_NO_PARK
constexpr bool kParkOn = false;
#else
constexpr bool kParkOn = true;
#endif
#ifdef RLB_NO_STAGE
constexpr bool kStageOn = false;
#else
constexpr bool kStageOn = true;
#endif
// dynamic shared memory of one block of nthr threads
constexpr size_t step_smem_bytes(int nthr, bool stage, int dim)
{
    return sizeof(f2) * size_t(nthr) * ((kParkOn ? kParkSlots : 0) + (stage ? 3 * dim * kStageBufs : 0));
}

// NP = 14: the 2-D symmetry reduction (DIM = 2, viscous step).  LIN: blocks
// of one row of 32 BY threads take consecutive cell pairs t of the x-fastest
// order (rows of ceil(nx / 2) pairs), for grids whose nx does not fill the
// tiles; otherwise blocks of 32 x BY threads take tiles of 64 x BY cells in
// one z-plane (the 1-D form: one row of tiles)
template <int DIM, bool EULER, bool VEC2, int LAT, int NP = 19, bool LIN = false, bool REC64 = false>
__global__ void __launch_bounds__(32 * RLB_F32_BY, VEC2 ? RLB_F32_MINB : 1)
    step_f32_kernel(const StepParams p, const float *__restrict__ f, const float *__restrict__ h,
                    float *__restrict__ fo, float *__restrict__ ho, float *__restrict__ prev)
{
    extern __shared__ f2 s_park[];
    int x0, y, z;
    if constexpr (LIN) {
        const unsigned ppr = unsigned(p.nx + 1) >> 1;
        const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
        const unsigned row = t / ppr;
        x0 = 2 * int(t - row * ppr);
        y = int(row % unsigned(p.ny));
        z = int(row / unsigned(p.ny));
        if (z >= p.nz) return;
    } else {
        unsigned bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
        if constexpr (DIM == 3) slab_order(p.slab_by, bx, by, bz);
        x0 = 2 * (bx * blockDim.x + threadIdx.x);
        y = by * blockDim.y + threadIdx.y;
        z = bz;
        if (x0 >= p.nx || y >= p.ny) return;
    }
    const long long ps = p.ps;

    Geo g;
    g.idx0 = x0 + p.nx * (y + p.ny * z);
    g.x0 = x0;
    g.has1 = x0 + 1 < p.nx;
    g.idx1 = g.has1 ? g.idx0 + 1 : g.idx0;
    g.oa = -2;
    g.oc = 2;
    g.xfix = 0u;
    if (VEC2) {
        if (x0 == 0) {   // x0-2, x0-1 are outside
            if (p.bc_lo[0] == BC_PERIODIC) g.oa = p.nx - 2;
            else { g.oa = 0; g.xfix |= p.bc_lo[0] == BC_OUTFLOW ? XF_LO_CLAMP : XF_LO_GHOST; }
        }
        if (x0 + 2 >= p.nx) {   // x0+2, x0+3 are outside
            if (p.bc_hi[0] == BC_PERIODIC) g.oc = -x0;
            else { g.oc = 0; g.xfix |= p.bc_hi[0] == BC_OUTFLOW ? XF_HI_CLAMP : XF_HI_GHOST; }
        }
    }
    {
        const int ds[4] = {-2, -1, 1, 2};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            bool gh;
            g.yoff[k] = DIM > 1 ? (map1(y + ds[k], p.ny, p.bc_lo[1], p.bc_hi[1], gh) - y) * p.nx : 0;
            g.zoff[k] = DIM > 2 ? (map1(z + ds[k], p.nz, p.bc_lo[2], p.bc_hi[2], gh) - z) * p.nx * p.ny : 0;
        }
    }
    if constexpr (DIM == 3) {
        g.sb[0] = 4u * unsigned(g.idx0 + g.oa);
        g.sb[1] = 4u * unsigned(g.idx0);
        g.sb[2] = 4u * unsigned(g.idx0 + g.oc);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            g.sb[3 + k] = 4u * unsigned(g.idx0 + g.yoff[k]);
            g.sb[7 + k] = 4u * unsigned(g.idx0 + g.zoff[k]);
        }
    }
    // threads per block as the launcher sets them (rlb_step_f32_launch.cuh), a
    // compile-time constant so that the shared-memory slots of this thread
    // sit at fixed offsets from one base address
    constexpr int nthr = (DIM == 1 && !LIN) ? 128 : 32 * RLB_F32_BY;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    constexpr bool STAGE = kStageOn && VEC2 && !EULER;
    update_pair<DIM, EULER, VEC2, LD_NC, kParkOn, STAGE, NP, LAT, REC64>(p, g, p.f_eta_over_s, p.f_kbulk, f, h, fo, ho,
                                                                  prev, ps,
                                                         s_park + tid, nthr,
                                                         s_park + (kParkOn ? kParkSlots * nthr : 0) + tid, nthr);
}

}  // namespace f32
}  // namespace rlb
