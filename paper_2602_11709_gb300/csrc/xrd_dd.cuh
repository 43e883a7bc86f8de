// Double-float ("dd") arithmetic for the accurate re-evaluation of weak
// reflections: a value is hi + lo with two FP32 numbers, about 48 significant
// bits. Built on the standard error-free transformations: Knuth's TwoSum,
// Dekker's Fast2Sum (|a| >= |b|) and the FMA form of Dekker's TwoProduct.
// FP32 throughput on this part is about 75 times its FP64 throughput, so a
// few dozen FP32 operations per dd step still beat one FP64 operation.
#pragma once

#include "xrd_internal.cuh"

namespace xrd {

struct DD {
    float hi, lo;
};

__device__ __forceinline__ DD dd_fast2sum(float a, float b)  // |a| >= |b| (or a == 0)
{
    const float s = a + b;
    return DD{s, b - (s - a)};
}

__device__ __forceinline__ DD dd_twosum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return DD{s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ DD dd_add(DD a, DD b)
{
    const DD s = dd_twosum(a.hi, b.hi);
    return dd_fast2sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ DD dd_neg(DD a) { return DD{-a.hi, -a.lo}; }

__device__ __forceinline__ DD dd_mul(DD a, DD b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return dd_fast2sum(p, e);
}

__device__ __forceinline__ DD dd_mul_f(DD a, float b)
{
    const float p = a.hi * b;
    const float e = fmaf(a.lo, b, fmaf(a.hi, b, -p));
    return dd_fast2sum(p, e);
}

// exact power-of-two scaling (no overflow or underflow checks: callers keep |k| small)
__device__ __forceinline__ DD dd_ldexp(DD a, int k) { return DD{ldexpf(a.hi, k), ldexpf(a.lo, k)}; }

// A double split into two floats: hi rounded to nearest, lo the rounded remainder.
__device__ __forceinline__ DD dd_from_double(double v)
{
    const float h = __double2float_rn(v);
    return DD{h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ double dd_to_double(DD a) { return (double)a.hi + (double)a.lo; }

// dd * 2^k for |k| <= 127 (results below 2^-126 become 0)
__device__ __forceinline__ DD dd_pow2(DD a, int k)
{
    if (k < -126) return DD{0.f, 0.f};
    const float sc = __int_as_float((127 + k) << 23);
    return DD{a.hi * sc, a.lo * sc};
}

// exp(-x) in double-float for x >= -80: x = n ln2/64 + r, |r| <= ln2/128, so
// exp(-x) = 2^-(n >> 6) 2^-((n & 63) / 64) exp(-r); ln2/64 in three parts
// (Cody and Waite: n * C1 is exact for |n| < 2^16), exp(-r) by its Taylor
// series to r^4 (next term below 4e-14). Relative error about 3e-10 (the
// rounding of r to one float). Results below 2^-126 are returned as 0.
__device__ __forceinline__ DD dd_exp_neg(DD x, const float2* __restrict__ tab)
{
    if (x.hi > 87.f) return DD{0.f, 0.f};
    constexpr float kInvL = 92.33248138427734f;  // 64 / ln 2
    constexpr float C1 = 0.01080322265625f, C2 = 2.720204065553844e-05f, C3 = -6.563933424574842e-13f;
    const float t = x.hi * kInvL + 12582912.f;  // round to nearest integer (1.5 * 2^23)
    const int n = __float_as_int(t) - 0x4B400000;
    const float nf = t - 12582912.f;
    float r = fmaf(-nf, C1, x.hi);
    r = fmaf(-nf, C2, r);
    r = fmaf(-nf, C3, r) + x.lo;
    // exp(-r) = (1 - r) + r^2 (1/2 - r/6 + r^2/24)
    const float p = r * r * fmaf(r, fmaf(r, 1.f / 24.f, -1.f / 6.f), 0.5f);
    DD e = dd_fast2sum(1.f, -r);
    e = dd_fast2sum(e.hi, e.lo + p);
    const float2 T = tab[n & 63];
    return dd_pow2(dd_mul(e, DD{T.x, T.y}), -(n >> 6));
}

// cos and sin of 2 pi P / 2^64: the nearest 1/256 turn from a table, the
// remainder |delta| <= pi/256 by its Taylor series (sin to delta^3, next term
// below 3e-12; cos to delta^4, next below 6e-15), combined by the angle sum.
__device__ __forceinline__ void dd_sincos_turn(unsigned long long P, const float4* __restrict__ tab, DD& c, DD& s)
{
    const unsigned long long k = (P + (1ull << 55)) >> 56;
    const long long d = (long long)(P - (k << 56));  // in [-2^55, 2^55): d 2^-64 turns
    const float4 T = tab[k & 255];
    const float th = (float)(int)(d >> 32) * 0x1p-32f;                  // exact: |d >> 32| < 2^23
    const float tl = (float)(unsigned)(d & 0xFFFFFFFFll) * 0x1p-64f;    // rounded below 2^-72 turn
    constexpr float P2h = 6.2831854820251465f, P2l = -1.7484555314695172e-07f;  // 2 pi
    const float p = th * P2h;
    float e = fmaf(th, P2h, -p);
    e = fmaf(th, P2l, e);
    e = fmaf(tl, P2h, e);
    const DD dl = dd_fast2sum(p, e);  // delta = 2 pi (th + tl)
    const float d2 = dl.hi * dl.hi;
    const DD sd{dl.hi, fmaf(-d2 * dl.hi, 1.f / 6.f, dl.lo)};  // sin(delta)
    const float cm = d2 * fmaf(-d2, 1.f / 24.f, 0.5f);       // 1 - cos(delta)
    // cos(t + delta) = C - (C cm + S sin delta)
    float q1 = T.z * sd.hi;
    float e1 = fmaf(T.z, sd.hi, -q1);
    e1 = fmaf(T.z, sd.lo, fmaf(T.w, sd.hi, e1));
    e1 = fmaf(T.x, cm, e1);
    c = dd_add(DD{T.x, T.y}, DD{-q1, -e1});
    // sin(t + delta) = S + (C sin delta - S cm)
    float q2 = T.x * sd.hi;
    float e2 = fmaf(T.x, sd.hi, -q2);
    e2 = fmaf(T.x, sd.lo, fmaf(T.y, sd.hi, e2));
    e2 = fmaf(-T.z, cm, e2);
    s = dd_add(DD{T.z, T.w}, DD{q2, e2});
}

}  // namespace xrd
