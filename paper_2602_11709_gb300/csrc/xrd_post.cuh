// Merge, family and sort-order helpers of the post-processing kernels (steps
// S4-S6), shared by the one-CTA-per-structure kernel (k_post.cu) and the flat
// passes of the largest structures (k_post_flat.cu).
#pragma once

#include "xrd_internal.cuh"

namespace xrd {

// 2-theta in degrees from |g|^2 in FP64, the definition 2 asin(lambda |g| / 2)
// with every step rounded on its own (no contraction), sin(theta) clamped at 1.
static __device__ __noinline__ double tt_deg64(double q, double lambda)
{
    double sth = __dmul_rn(__dmul_rn(lambda, __dsqrt_rn(q)), 0.5);
    if (sth > 1.0) sth = 1.0;
    return __dmul_rn(__dmul_rn(2.0, asin(sth)), 180.0 / kPi);
}

// Merge test: 2theta(qb) - 2theta(qa) < tol for qb >= qa > 0. With
// x = lambda sqrt(q) / 2 = sin theta and c = cos theta,
// tan((2theta_b - 2theta_a) / 4) = (xb - xa) / (ca + cb) and
// xb - xa = (lambda / 2)(qb - qa) / (sqrt qa + sqrt qb); qb - qa is exact in FP64
// for close values. Comparing against ttol = tan(tol / 4) (tol in radians)
// leaves neither a division nor an arctangent. This FP32 form is good to about
// 1e-6 relative, plus the rounding of 1 - lambda^2 q / 4 relative to cos^2(theta)
// (~1.3e-7 / cos^2); a pair within 1e-5 + 1e-6 / cos^2 of the tolerance is
// decided in FP64 from the definition instead, so that every merge decision is
// an FP64 one. It is the same decision as a CPU evaluation of the definition
// except for gaps within a few ulp of 2-theta of the tolerance: CUDA's asin
// and the C library's asin are each accurate to about an ulp but are not
// guaranteed to round alike, so such a gap may fall on either side.
static __device__ __forceinline__ bool tt_close(double qa, double qb, float l2, float lh, float ttol, double lambda,
                                         double tol)
{
    if (dbits(qb) <= dbits(qa)) return ttol > 0.f;  // equal |g|^2: a gap of 0
    if (ttol == INFINITY) return true;              // tol above 180 degrees: every gap is below it
    const float dqf = d2f_pos(qb - qa);
    const float qaf = d2f_pos(qa), qbf = d2f_pos(qb);
    const float ua = fmaxf(fmaf(-l2, qaf, 1.f), 1e-30f), ub = fmaxf(fmaf(-l2, qbf, 1.f), 1e-30f);
    const float sq = qaf * rsqrtf(qaf) + qbf * rsqrtf(qbf);
    const float c = ua * rsqrtf(ua) + ub * rsqrtf(ub);
    const float lhs = lh * dqf, rhs = ttol * (sq * c);
    const float band = fmaf(1e-6f, __frcp_rn(fminf(ua, ub)), 1e-5f);
    if (!(fabsf(lhs - rhs) <= band * rhs)) return lhs < rhs;
    return __dsub_rn(tt_deg64(qb, lambda), tt_deg64(qa, lambda)) < tol;
}

// Family key: the absolute values of the indices sorted descending, packed:
// (h, k, l) and a 0, or for a hexagonal cell the Miller-Bravais (h, k, i = -h - k, l)
// (|i| <= 1022 fits the 10-bit fields). Families are the classes of equal keys.
static __device__ __forceinline__ unsigned long long family_key(uint32_t key, bool hex)
{
    const int h = hkl_h(key), k = hkl_k(key);
    int v0 = abs(h), v1 = abs(k), v2 = abs(hkl_l(key)), v3 = hex ? abs(h + k) : 0, t;
    // sorting network for 4 values, descending
    if (v1 > v0) { t = v0; v0 = v1; v1 = t; }
    if (v3 > v2) { t = v2; v2 = v3; v3 = t; }
    if (v2 > v0) { t = v0; v0 = v2; v2 = t; }
    if (v3 > v1) { t = v1; v1 = v3; v3 = t; }
    if (v2 > v1) { t = v1; v1 = v2; v2 = t; }
    return ((unsigned long long)v0 << 30) | ((unsigned long long)v1 << 20) | ((unsigned long long)v2 << 10) |
           (unsigned long long)v3;
}

// Family key under a caller's point group (the symmetry-aware mode): the family
// of g is its orbit {M g, -M g} over the group's operations M (Friedel's law adds
// the inversion); the key is the orbit's lexicographically largest member,
// packed in 12-bit fields (operations have entries in {-1, 0, 1}, so an image of
// an index within +-511 stays within +-1533).
static __device__ __forceinline__ unsigned long long pg_pack(int a, int b, int c)
{
    return ((unsigned long long)(a + 2048) << 24) | ((unsigned long long)(b + 2048) << 12) |
           (unsigned long long)(c + 2048);
}
static __device__ __forceinline__ unsigned long long pg_family_key(uint32_t key, const int8_t* __restrict__ ops,
                                                                   int n)
{
    const int h = hkl_h(key), k = hkl_k(key), l = hkl_l(key);
    unsigned long long best = max(pg_pack(h, k, l), pg_pack(-h, -k, -l));
    for (int m = 0; m < n; m++) {
        const int8_t* M = ops + 9 * m;
        const int x = M[0] * h + M[1] * k + M[2] * l, y = M[3] * h + M[4] * k + M[5] * l,
                  z = M[6] * h + M[7] * k + M[8] * l;
        best = max(best, max(pg_pack(x, y, z), pg_pack(-x, -y, -z)));
    }
    return best;
}

// number of distinct families among the members i0..i1-1 of one peak; fk(i): the family key of member i
template <typename FK>
static __device__ __forceinline__ int count_families(FK fk, int i0, int i1)
{
    int nfam = 0;
    for (int i = i0; i < i1; i++) {
        const unsigned long long k = fk(i);
        bool lead = true;
        for (int j = i0; j < i && lead; j++) lead = fk(j) != k;
        nfam += lead;
    }
    return nfam;
}

// sort order: ascending |g|^2, ties by descending (h, k, l)
static __device__ __forceinline__ bool before(double qa, uint32_t ka, double qb, uint32_t kb)
{
    const unsigned long long a = dbits(qa), b = dbits(qb);  // q > 0: bit order is numeric order
    return a < b || (a == b && ka > kb);
}

}  // namespace xrd
