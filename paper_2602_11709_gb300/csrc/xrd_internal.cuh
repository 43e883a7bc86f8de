// Internal types and device helpers of the GB300 powder-XRD engine.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "xrd.h"

namespace xrd {

constexpr double kPi = 3.14159265358979323846;
// cos^2(theta) at theta = 90 degrees as FP64 evaluates it (cos of the double nearest pi/2,
// squared): the floor of cos^2 theta, so that a reflection on the 2theta = 180 degrees
// surface gets a large finite Lorentz factor instead of a division by zero.
constexpr double kCos90Sq = 3.749399456654644e-33;
constexpr double kFScale = 41.78214;  // Mott-Bethe factor 8 pi^2 a0 of f(s) (Sec. 1, atomic scattering factors)
constexpr int kZmaxLimit = 255;
constexpr int kHklLimit = 511;        // |h|, |k|, |l| fit the 10-bit fields of the packed key
// Post-processing size classes: structures with at most kPostCap[c] reflections
// (held in shared memory, 35 B per reflection) go to class c, one CTA each with
// 64, 128, 192, 256, 256, 512, 512 or 1024 threads; finer classes at the small
// end keep the shared memory of a CTA close to what its structure needs, so
// more structures are in flight per SM. Larger structures go to the last
// class, processed by flat device-wide passes (k_post_flat.cu). Every class
// runs on a stream of its own.
constexpr int kPostClasses = 9;
constexpr int kRunsPerTile = 32;  // structure-factor tile: one run of reflections per lane of a warp
constexpr int kPostCap0 = 256, kPostCap1 = 512, kPostCap2 = 768, kPostCap3 = 1024, kPostCap4 = 1536,
              kPostCap5 = 2048, kPostCap6 = 3072, kPostCap7 = 6144;
constexpr int kPostFlatClass = kPostClasses - 1;
constexpr int kPostStreams = kPostClasses;
__host__ __device__ __forceinline__ int post_class(long long c)
{
    return c <= kPostCap0   ? 0
           : c <= kPostCap1 ? 1
           : c <= kPostCap2 ? 2
           : c <= kPostCap3 ? 3
           : c <= kPostCap4 ? 4
           : c <= kPostCap5 ? 5
           : c <= kPostCap6 ? 6
           : c <= kPostCap7 ? 7
                            : 8;
}
// Flag words of a call (ints of the zeroed flags area): the class counts and the classes' work counters.
constexpr int kFlagClsCnt = 32, kFlagClsNext = 48, kFlagPfBar = 4;

// Per-structure geometry written by k_prep (step S0).
struct Geo {
    double gs[6];  // reciprocal metric G* stored as (11, 22, 33, 12, 13, 23)
    double g2[3];  // 2 G*12, 2 G*13, 2 G*23 (exact doubles of the off-diagonal terms)
    float gf[6];   // G* rounded to FP32, for the enumeration filter
    float gl[6];   // G* - gf (the low words of a two-float G*; off-diagonals doubled in hi and lo below)
    int H, K, L;   // enumeration box |h| <= H ...
    int status;    // XRD_OK or XRD_EINVAL
    int hex;       // 1: hexagonal cell (alpha, beta within 5 deg of 90, gamma within 5 deg of 120,
                   // |a - b| < 0.01 A): families by Miller-Bravais indices
};

// Atom record for the FP32 structure-factor loops (sorted by element within a
// structure); 32 bytes, read as two 16-byte shared-memory loads.
struct __align__(16) Atom32 {
    uint32_t X, Y, Z;  // coordinates in 32-bit fixed point: round(x * 2^32) mod 2^32
    float nb;          // -B * log2(e): exp(-B s^2) = 2^(nb s^2)
    float lo;          // log2(occ): occ folds into the same exp2
    int32_t z;         // element number
    int32_t src;       // index of the atom within its structure in the caller's order
    float zf;          // element number as a float (f(s) = Z + ...)
};

// Atom record for the FP64 loops and the FP64 phase.
struct __align__(16) Atom64 {
    double x, y, z, B, occ;
    int32_t zz, pad;
};

// f(s) = Z + s^2 sum_i a'_i 2^(bl_i s^2) with a'_i = -41.78214 a_i, bl_i = -b_i log2(e).
struct __align__(16) Coef32 {
    float a[4];
    float bl[4];
};

// Atom record of the accurate re-evaluation (k_refine), element-sorted like
// Atom32: coordinates in 64-bit fixed point, occupancy and B as two floats.
struct __align__(16) AtomR {
    unsigned long long X, Y, Z;  // round(x * 2^64) mod 2^64
    float oh, ol;                // occupancy = oh + ol
    float bh, bl;                // B = bh + bl (angstrom^2)
    int32_t z;                   // element number
    int32_t pad;
};

// round(v * 2^64) mod 2^64 for a finite double, by bit arithmetic (ties round up).
__device__ __forceinline__ unsigned long long fix64(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FFull);
    if (e == 0) return 0ull;  // zero or subnormal: below 2^-1022
    const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int sh = e - 1075 + 64;  // v * 2^64 = +-m * 2^sh
    unsigned long long r;
    if (sh >= 64) r = 0ull;
    else if (sh >= 0) r = m << sh;
    else if (sh > -64) r = (m >> (-sh)) + ((m >> (-sh - 1)) & 1ull);
    else r = 0ull;
    return (b >> 63) ? 0ull - r : r;
}

// Reflection key: (h + 512, k + 512, l + 512) in three 10-bit fields, so that
// the unsigned order of keys is the lexicographic order of signed (h, k, l).
__host__ __device__ __forceinline__ uint32_t hkl_pack(int h, int k, int l)
{
    return ((uint32_t)(h + 512) << 20) | ((uint32_t)(k + 512) << 10) | (uint32_t)(l + 512);
}
__host__ __device__ __forceinline__ int hkl_h(uint32_t p) { return (int)((p >> 20) & 1023u) - 512; }
__host__ __device__ __forceinline__ int hkl_k(uint32_t p) { return (int)((p >> 10) & 1023u) - 512; }
__host__ __device__ __forceinline__ int hkl_l(uint32_t p) { return (int)(p & 1023u) - 512; }

// Positive normal double -> float by bit arithmetic (truncation). The hardware
// conversion unit is slow on this part; callers use it only for values that
// are positive, normal and in float range.
__device__ __forceinline__ float d2f_pos(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    return __uint_as_float(((hi - (896u << 20)) << 3) | (lo >> 29));
}

// Float (finite, any sign, zero or normal) -> double by bit arithmetic; denormals become 0.
__device__ __forceinline__ double f2d_fast(float x)
{
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    const uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu);
    const uint32_t lo = u << 29;
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

// round(v * 2^32) mod 2^32 for |v| < 2^19: adding 1.5 * 2^20 puts 2^-32 at the
// last mantissa bit, so the low word of the sum is the wrapped fixed-point value.
__device__ __forceinline__ uint32_t fix32(double v)
{
    const double t = __dadd_rn(v, 1572864.0);
    return (uint32_t)(unsigned long long)__double_as_longlong(t);
}

// ---- programmatic dependent launch ----
// Every kernel starts with pdl_enter(): it waits until the grid it depends on
// has completed and its memory is visible (a no-op when the kernel was launched
// the ordinary way), then lets the next grid on the stream be launched, so that
// grid's launch and rasterisation overlap this one's execution. A dependent
// grid can start only once every CTA of this grid is resident, and it waits in
// its own pdl_enter(), so the order of the stream is kept.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch k on st as a programmatic dependent of the previous kernel on st.
template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<P>(args)...);
}

// ---- two-float ("double-float") arithmetic: value = hi + lo, |lo| <= ulp(hi) / 2 ----
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 f2_quick(float a, float b)  // |a| >= |b|
{
    const float s = a + b;
    return F2{s, b - (s - a)};
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb) + (a.lo + b.lo);
    return f2_quick(s, e);
}
// a * n for an integer n exactly representable in FP32
__device__ __forceinline__ F2 f2_mul_int(F2 a, float n)
{
    const float p = a.hi * n;
    const float e = fmaf(a.hi, n, -p) + a.lo * n;
    return f2_quick(p, e);
}

// Exact int -> double by bit assembly (|v| < 2^31); keeps the conversion off
// the FP64 unit, which this part has little of.
__device__ __forceinline__ double i2d_exact(int v)
{
    if (v == 0) return 0.0;
    const unsigned long long sign = v < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned a = v < 0 ? (unsigned)(-v) : (unsigned)v;
    const int e = 31 - __clz(a);
    const unsigned long long m = ((unsigned long long)a << (52 - e)) & 0x000FFFFFFFFFFFFFull;
    return __longlong_as_double((long long)(sign | ((unsigned long long)(1023 + e) << 52) | m));
}

// Order of non-negative doubles through their bit patterns (integer compare).
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sin and cos of 2 pi P / 2^32 (P an exact phase in turns, 32-bit fixed point) on the FMA pipe:
// the nearest quarter turn q comes from the top bits (exact), the remainder d = P - q 2^30 in
// [-2^29, 2^29) gives a = 2 pi d / 2^32 in [-pi/4, pi/4), and polynomials in a^2 fitted to sin and
// cos on that interval (least squares on Chebyshev nodes with Lawson reweighting, coefficients
// rounded to FP32; approximation error below 2.3e-9) are rotated back by q quarter turns. About
// 2e-8 RMS and 1e-7 largest absolute error, five times below the SFU's sin/cos, whose error
// dominated the FP32 structure factor.
__device__ __forceinline__ void sincos_turn32(uint32_t P, float& s, float& c)
{
    const uint32_t q = (P + 0x20000000u) >> 30;
    const float a = (float)(int32_t)(P - (q << 30)) * 1.4629180792671596e-09f;  // 2 pi / 2^32
    const float a2 = a * a;
    const float ps = fmaf(fmaf(-0.00019495634478516877f, a2, 0.00833197869360447f), a2, -0.16666650772094727f);
    const float sa = fmaf(a * a2, ps, a);
    const float pc = fmaf(fmaf(fmaf(2.439044874336105e-05f, a2, -0.0013886763481423259f), a2, 0.04166662320494652f),
                          a2, -0.5f);
    const float ca = fmaf(a2, pc, 1.f);
    const bool swap = q & 1u;  // (sin, cos)(a + q pi/2): q = 1: (cos, -sin), 2: (-sin, -cos), 3: (-cos, sin)
    const float s1 = swap ? ca : sa, c1 = swap ? sa : ca;
    s = __int_as_float(__float_as_int(s1) ^ (int)((q & 2u) << 30));
    c = __int_as_float(__float_as_int(c1) ^ (int)(((q + 1u) & 2u) << 30));
}

// Positive normal double -> two floats, q = qh + ql to about 2^-47 relative,
// by bit arithmetic only: qh is q truncated to 24 significant bits, ql holds the
// next 23 bits (built exactly in the mantissa of 2^23 and scaled by a power of
// two; it becomes 0 when q < 2^-80).
__device__ __forceinline__ void split_pos(double q, float& qh, float& ql)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(q);
    qh = d2f_pos(q);
    const uint32_t rest = (uint32_t)b & 0x1FFFFFFFu;  // significand bits below qh's
    const int e = (int)((uint32_t)(b >> 52) & 0x7FFu) - 1023;
    const float m = __int_as_float(0x4B000000 | (rest >> 6)) - 8388608.f;
    ql = m * __int_as_float(max(e + 81, 0) << 23);  // weight of bit 6 of rest: 2^(e - 46)
}

// ---- 2-theta of a reflection from |g|^2 without FP64 arithmetic but one addition ----
// theta in [0, pi/4] is found from a table at theta_j = j * pi / 4096 (2theta_j =
// j * 360 / 4096 degrees, exact in binary) and FP32 Newton steps on the small
// remainder u = 2 (theta - theta_j); angles above 45 degrees use the complement
// (sin^2 theta = 1 - sin^2(90 deg - theta)). sin^2 theta = q lambda^2 / 4 and the
// table's sin^2 theta_j are carried as two floats, so the remainder is exact to
// about 1e-14. Error about 1e-8 degrees.
constexpr int kTabN = 1024;
constexpr float kTabStepDeg = 360.f / 4096.f;  // 2theta spacing of the table (exact)
struct __align__(16) TTab {
    float Sh, Sl;  // sin^2 theta_j as two floats
    float A;       // sin 2 theta_j
    float Bc;      // cos 2 theta_j
};

// 2theta in degrees for |g|^2 = q (> 0, normal) and lambda^2 / 4 = Lh + Ll;
// sin^2 theta above 1 is taken as 1 (90 degrees theta).
__device__ __forceinline__ double two_theta_q(double q, float Lh, float Ll, const TTab* __restrict__ tab)
{
    float qh, ql;
    split_pos(q, qh, ql);
    // X = q L as two floats
    float Xh = qh * Lh;
    float Xl = fmaf(qh, Lh, -Xh) + fmaf(qh, Ll, ql * Lh);
    if (Xh > 1.f || (Xh == 1.f && Xl > 0.f)) {
        Xh = 1.f;
        Xl = 0.f;
    }
    const bool comp = Xh > 0.5f || (Xh == 0.5f && Xl > 0.f);
    const float Yh = comp ? 1.f - Xh : Xh;  // exact for Xh in [0.5, 1]
    const float Yl = comp ? -Xl : Xl;
    const float Yf = Yh + Yl;
    const float th0 = asinf(sqrtf(fmaxf(Yf, 0.f)));
    int j = __float2int_rn(th0 * (float)(4.0 * kTabN / kPi));
    j = min(max(j, 0), kTabN);
    float T, v;  // 2theta = T + v with T a multiple of the table step (exact in float)
    if (j <= 2) {
        T = 0.f;
        v = th0 * (float)(360.0 / kPi);
    } else {
        const TTab e = tab[j];
        const float r = (Yh - e.Sh) + (Yl - e.Sl);
        float u = 4.f * r / (e.A + sqrtf(fmaf(4.f * e.Bc, r, e.A * e.A)));
#pragma unroll
        for (int it = 0; it < 2; it++) {
            const float u2 = u * u;
            const float su = u - u * u2 * (1.f / 6.f);
            const float cu = u2 * (0.5f - u2 * (1.f / 24.f));
            const float fv = fmaf(e.A, su, fmaf(e.Bc, cu, -2.f * r));
            const float fp = fmaf(e.A, 1.f - 0.5f * u2, e.Bc * su);
            u -= fv / fp;
        }
        T = (float)j * kTabStepDeg;
        v = u * (float)(180.0 / kPi);
    }
    if (comp) {
        T = 180.f - T;  // exact: both are multiples of 45 / 512
        v = -v;
    }
    return f2d_fast(T) + f2d_fast(v);
}

// d = 1/sqrt(q) for q > 0 in float range: an FP32 seed refined by one Newton
// step whose residual 1 - q y0^2 is formed exactly in FP32 (q split into two
// floats, y0^2 into two floats); about 1e-13 relative, one FP64 addition.
__device__ __forceinline__ double inv_sqrt_df(double q)
{
    float qh, ql;
    split_pos(q, qh, ql);
    const float y0 = rsqrtf(qh);
    const float p = y0 * y0, pe = fmaf(y0, y0, -p);
    float r = fmaf(-qh, p, 1.f);
    r = fmaf(-qh, pe, fmaf(-ql, p, r));
    return f2d_fast(y0) + f2d_fast(0.5f * y0 * r * fmaf(0.75f, r, 1.f));
}

// ---- block-wide primitives over generic pointers (shared or global memory) ----

__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive prefix sum of a[0..n) in place by the whole block; returns the
// total. `tmp` is shared scratch of at least 33 ints. All threads must call.
// In-place exclusive scan of a[0..n) in shared memory by the whole block; each
// thread takes one contiguous segment, so the block synchronises three times
// whatever n is. Returns the total. tmp: 33 ints of shared memory.
__device__ __forceinline__ int block_excl_scan(int* a, int n, int* tmp)
{
    const int nt = blockDim.x, nw = (nt + 31) >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int seg = (n + nt - 1) / nt;
    const int i0 = min((int)threadIdx.x * seg, n), i1 = min(i0 + seg, n);
    int s = 0;
    for (int i = i0; i < i1; i++) s += a[i];
    const int inc = warp_incl_scan(s);
    if (lane == 31) tmp[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int v = lane < nw ? tmp[lane] : 0;
        const int si = warp_incl_scan(v);
        if (lane < nw) tmp[lane] = si - v;
        if (lane == 31) tmp[32] = si;
    }
    __syncthreads();
    int run = tmp[w] + inc - s;
    const int total = tmp[32];
    for (int i = i0; i < i1; i++) {
        const int v = a[i];
        a[i] = run;
        run += v;
    }
    __syncthreads();
    return total;
}

// Two exclusive scans of the same length at once (a and b); totals in ta, tb.
// tmp: 66 ints of shared memory.
__device__ __forceinline__ void block_excl_scan2(int* a, int* b, int n, int* tmp, int& ta, int& tb)
{
    const int nt = blockDim.x, nw = (nt + 31) >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int seg = (n + nt - 1) / nt;
    const int i0 = min((int)threadIdx.x * seg, n), i1 = min(i0 + seg, n);
    int sa = 0, sb = 0;
    for (int i = i0; i < i1; i++) {
        sa += a[i];
        sb += b[i];
    }
    const int ia = warp_incl_scan(sa), ib = warp_incl_scan(sb);
    if (lane == 31) {
        tmp[w] = ia;
        tmp[33 + w] = ib;
    }
    __syncthreads();
    if (w == 0) {
        const int va = lane < nw ? tmp[lane] : 0, vb = lane < nw ? tmp[33 + lane] : 0;
        const int xa = warp_incl_scan(va), xb = warp_incl_scan(vb);
        if (lane < nw) {
            tmp[lane] = xa - va;
            tmp[33 + lane] = xb - vb;
        }
        if (lane == 31) {
            tmp[32] = xa;
            tmp[65] = xb;
        }
    }
    __syncthreads();
    int ra = tmp[w] + ia - sa, rb = tmp[33 + w] + ib - sb;
    ta = tmp[32];
    tb = tmp[65];
    for (int i = i0; i < i1; i++) {
        const int va = a[i], vb = b[i];
        a[i] = ra;
        b[i] = rb;
        ra += va;
        rb += vb;
    }
    __syncthreads();
}

// Exclusive block-wide prefix of one 64-bit value per thread (two barriers;
// ws: 33 long longs of shared memory, free again on return). Returns this
// thread's exclusive prefix; *total gets the block total.
__device__ __forceinline__ long long block_prefix_ll(long long v, long long* ws, long long* total)
{
    const int nw = (blockDim.x + 31) >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        const long long x = lane < nw ? ws[lane] : 0;
        long long y = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        if (lane < nw) ws[lane] = y - x;
        if (lane == 31) ws[32] = y;
    }
    __syncthreads();
    const long long r = ws[w] + inc - v;
    *total = ws[32];
    __syncthreads();
    return r;
}

// Exclusive scan of one chunk of ITEMS * blockDim values held as v[u] for
// element u * blockDim + tid (the coalesced order they were loaded in):
// transposed through buf (ITEMS * blockDim long longs of shared memory) so
// that each thread scans ITEMS consecutive elements, then back. v receives the
// exclusive prefixes in the same order; *total the chunk's total.
template <int kScanItems>
__device__ __forceinline__ void chunk_scan(long long (&v)[kScanItems], long long* buf, long long* ws, long long* total)
{
    const int nt = blockDim.x, tid = threadIdx.x;
#pragma unroll
    for (int u = 0; u < kScanItems; u++) buf[u * nt + tid] = v[u];
    __syncthreads();
    long long loc[kScanItems], sum = 0;
#pragma unroll
    for (int u = 0; u < kScanItems; u++) {
        loc[u] = buf[tid * kScanItems + u];
        sum += loc[u];
    }
    long long run = block_prefix_ll(sum, ws, total);
#pragma unroll
    for (int u = 0; u < kScanItems; u++) {
        buf[tid * kScanItems + u] = run;
        run += loc[u];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kScanItems; u++) v[u] = buf[u * nt + tid];
    __syncthreads();
}

__device__ __forceinline__ double block_max_double(double v, double* tmp)
{
    const int nw = (blockDim.x + 31) >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) tmp[w] = v;
    __syncthreads();
    double r = tmp[0];
    for (int i = 1; i < nw; i++) r = fmax(r, tmp[i]);
    __syncthreads();
    return r;
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* tmp)
{
    const int nw = (blockDim.x + 31) >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, (unsigned long long)__shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) tmp[w] = v;
    __syncthreads();
    unsigned long long r = tmp[0];
    for (int i = 1; i < nw; i++) r = max(r, tmp[i]);
    __syncthreads();
    return r;
}

__device__ __forceinline__ int block_sum_int(int v, int* tmp)
{
    const int nw = (blockDim.x + 31) >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) tmp[w] = v;
    __syncthreads();
    int r = 0;
    for (int i = 0; i < nw; i++) r += tmp[i];
    __syncthreads();
    return r;
}

}  // namespace xrd
