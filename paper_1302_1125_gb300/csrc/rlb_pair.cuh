// rlb_pair.cuh -- two-cell arithmetic for the FP32-storage step.
//
// One thread updates two x-adjacent cells.  Every per-cell quantity is held
// as a pair (cell x0, cell x0 + 1) and the arithmetic both cells perform
// identically is issued as packed FP32x2 instructions (add/sub/mul/fma.f32x2,
// sm_100 and later), which halves the instruction count of that work.
#pragma once

#include <cuda_runtime.h>

namespace rlb {

struct __align__(8) f2 {
    float x, y;
};

__device__ __forceinline__ unsigned long long pk(f2 a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ f2 upk(unsigned long long r)
{
    f2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ f2 mk(float a, float b) { return f2{a, b}; }
__device__ __forceinline__ f2 bc(float a) { return f2{a, a}; }

__device__ __forceinline__ f2 operator+(f2 a, f2 b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
    return upk(r);
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
    return upk(r);
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
    return upk(r);
}
// a * b + c, one rounding
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
    return upk(r);
}
__device__ __forceinline__ f2 operator-(f2 a) { return f2{-a.x, -a.y}; }

// minmod(a, b) (Eq. 53): the smaller magnitude when a and b share a sign,
// zero otherwise.  min.xorsign.abs gives m = min(|a|, |b|) carrying the sign
// sign(a) xor sign(b): m > 0 exactly when the signs agree, then the result is
// m with the sign of a; otherwise max(m, 0) = 0.
#ifndef RLB_MM_MEDIAN
__device__ __forceinline__ float mm(float a, float b)
{
    float m;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(m) : "f"(a), "f"(b));
    return copysignf(fmaxf(m, 0.0f), a);
}
#else
__device__ __forceinline__ float mm(float a, float b)
{
    return fminf(fmaxf(a, b), fmaxf(fminf(a, b), 0.0f));   // median(0, a, b)
}
#endif
__device__ __forceinline__ f2 mm(f2 a, f2 b) { return f2{mm(a.x, b.x), mm(a.y, b.y)}; }

// ---------------------------------------------------------------------------
// Double-float (unevaluated sum hi + lo) accumulation, error-free in FP32:
// Knuth's TwoSum gives s + e = a + b exactly.
// ---------------------------------------------------------------------------
struct df2 {
    f2 hi, lo;
};

__device__ __forceinline__ void two_sum(f2 a, f2 b, f2 &s, f2 &e)
{
    s = a + b;
    const f2 bb = s - a;
    const f2 aa = s - bb;
    e = (a - aa) + (b - bb);
}

__device__ __forceinline__ void acc(df2 &d, f2 v)
{
    f2 s, e;
    two_sum(d.hi, v, s, e);
    d.hi = s;
    d.lo = d.lo + e;
}

// a^2 as a double-float from a double-float a (product error-free via FMA)
__device__ __forceinline__ df2 sq(const df2 &a)
{
    const f2 p = a.hi * a.hi;
    f2 e = fma2(a.hi, a.hi, -p);
    e = fma2(a.hi + a.hi, a.lo, e);
    df2 r;
    two_sum(p, e, r.hi, r.lo);
    return r;
}

// a + b of double-floats, result renormalised
__device__ __forceinline__ df2 dadd(const df2 &a, const df2 &b)
{
    f2 s, e;
    two_sum(a.hi, b.hi, s, e);
    e = e + (a.lo + b.lo);
    df2 r;
    two_sum(s, e, r.hi, r.lo);
    return r;
}

// c * a for a double-float constant c = ch + cl
__device__ __forceinline__ df2 dscale(const df2 &a, float ch, float cl)
{
    const f2 p = bc(ch) * a.hi;
    f2 e = fma2(bc(ch), a.hi, -p);
    e = fma2(bc(cl), a.hi, e);
    e = fma2(bc(ch), a.lo, e);
    df2 r;
    two_sum(p, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df2 dneg(const df2 &a) { return df2{-a.hi, -a.lo}; }

}  // namespace rlb
