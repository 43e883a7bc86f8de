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

}  // namespace xrd
