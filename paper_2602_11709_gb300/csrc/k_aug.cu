// Augmented pattern: the experimental effects that synthetic training patterns
// for ML models carry (Sec. 1: peak broadening, noise, preferred orientation),
// applied on the GPU to the structure factors of the pattern path.
//
//   y_k = sum_g 2 I_g P_g PV(t_k - 2theta_g)   (Friedel-unique g; g and -g share I, P, 2theta)
//   P_g = (r^2 c + (1 - c) / r)^(-3/2),  c = cos^2 of the angle between g and n (metric G*)
//   PV(u) = eta (2 / (pi w)) / (1 + x^2) + (1 - eta) (2 / w) sqrt(ln 2 / pi) 2^(-x^2),  x = 2 u / w
//   then y_k += sigma sqrt(max(y_k, 0)) z_k.
//
// k_aug_order lists the structures by reflection count, largest first.
// k_aug_sum gives each CTA 1024 grid points of one structure (kAugPts
// consecutive points per thread) and streams all of the structure's reflections
// through shared memory, turning each into a record as it is staged: its grid
// cell b, the offset d of 2theta within the cell scaled by s = 2 dt / w, and the
// Lorentzian and Gaussian amplitudes. The Lorentzian has no window: every
// (point, reflection) pair costs half a reciprocal (MUFU, one per pair of
// points) and about five FP32 operations. The Gaussian is evaluated by a warp
// only for the reflections that reach its points with x^2 < 40 (a test made
// once per reflection while staging).
//
// Precision: x = (k - b) s - d s with k - b an exact integer in FP32 (|k|, |b| <
// 2^22); for s <= 1 the points after a thread's first take x + j s (absolute
// error a few ulp of kAugPts s there); sums are FP32 in reflection order.
#include <cmath>

#include "xrd_internal.cuh"
#include "xrd_launch.h"

namespace xrd {

constexpr int kAugPts = 8;                       // consecutive grid points per thread
constexpr int kAugThreads = 1024 / kAugPts;
constexpr int kAugSpan = kAugThreads * kAugPts;  // grid points per CTA
constexpr int kAugWarps = kAugThreads / 32;
constexpr int kAugBuckets = 128;                 // reflection-count buckets of the largest-first order
constexpr int kAugChunk = 1024;                  // reflections staged in shared memory at a time

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Structures by reflection count, largest first (buckets of a quarter octave),
// so that the CTAs of the largest structures start first. One CTA.
__global__ void __launch_bounds__(1024) k_aug_order(const AugArgs a)
{
    pdl_enter();
    __shared__ int cnt[kAugBuckets];
    for (int i = threadIdx.x; i < kAugBuckets; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    auto bucket = [&](int s) {
        const int64_t R = a.refl_off[s + 1] - a.refl_off[s];
        return R <= 0 ? 0 : min(kAugBuckets - 1, 1 + (int)(4.f * log2f((float)R)));
    };
    for (int s = threadIdx.x; s < a.n_struct; s += blockDim.x) atomicAdd(&cnt[bucket(s)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = kAugBuckets - 1; b >= 0; b--) {
            const int c = cnt[b];
            cnt[b] = acc;
            acc += c;
        }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < a.n_struct; s += blockDim.x) a.aorder[atomicAdd(&cnt[bucket(s)], 1)] = s;
}

// Per-structure constants of the profile sum (all zero for a structure that is
// invalid or has invalid effect parameters: no reflections, a zero row).
struct AugStruct {
    int n;             // reflections summed
    int valid, lor, gau, po;
    float sc;          // 2 dt / fwhm
    float cl, cg;      // Lorentzian and Gaussian prefactors of the area-normalised profile
    float m0, m1, m2;  // G* n / |n| (|n| in the metric G*): g.n / |n| = h m0 + k m1 + l m2
    float r;           // March-Dollase r
    float sig;         // noise scale
};

// Validates the effect parameters of structure s (every comparison is false
// for NaN, so NaN parameters fail). bad_params: the structure itself is valid
// but its parameters are not.
__device__ AugStruct aug_struct(const AugArgs& a, int s, bool& bad_params)
{
    AugStruct c{};
    const bool geo_ok = !*a.abort_flag && a.geo[s].status == XRD_OK;
    const double w = a.fwhm[s], eta = a.eta[s];
    const double sc = 2.0 * a.dt / w;
    bool ok = w > 0.0 && w <= 1e6 && sc <= 1e6 && eta >= 0.0 && eta <= 1.0;
    double M0 = 0.0, M1 = 0.0, M2 = 0.0, nn = 1.0, R = 1.0, sig = 0.0;
    if (a.po_dir && geo_ok) {
        const double* n = a.po_dir + 3 * (int64_t)s;
        const double* g = a.geo[s].gs;
        R = a.po_r[s];
        M0 = g[0] * n[0] + g[3] * n[1] + g[4] * n[2];
        M1 = g[3] * n[0] + g[1] * n[1] + g[5] * n[2];
        M2 = g[4] * n[0] + g[5] * n[1] + g[2] * n[2];
        nn = n[0] * M0 + n[1] * M1 + n[2] * M2;
        ok = ok && R >= 1e-6 && R <= 1e6 && nn > 0.0 && nn < INFINITY && fabs(M0) < INFINITY &&
             fabs(M1) < INFINITY && fabs(M2) < INFINITY;
    }
    if (a.noise_z) {
        sig = a.noise_sigma[s];
        ok = ok && sig >= 0.0 && sig < INFINITY;
    }
    bad_params = geo_ok && !ok;
    if (!(geo_ok && ok)) return c;
    c.n = (int)(a.refl_off[s + 1] - a.refl_off[s]);
    c.valid = 1;
    c.lor = eta > 0.0;
    c.gau = eta < 1.0;
    c.sc = (float)sc;
    c.cl = (float)(eta * 2.0 / (kPi * w));
    c.cg = (float)((1.0 - eta) * (2.0 / w) * sqrt(log(2.0) / kPi));
    c.po = a.po_dir != nullptr;
    const double inv = 1.0 / sqrt(nn);
    c.m0 = (float)(M0 * inv);
    c.m1 = (float)(M1 * inv);
    c.m2 = (float)(M2 * inv);
    c.r = (float)R;
    c.sig = (float)sig;
    return c;
}

// Record of reflection j: (-b, -d s, Lorentzian amplitude, Gaussian amplitude).
__device__ __forceinline__ float4 aug_record(const AugArgs& a, const AugStruct& c, int64_t j)
{
    const double q = a.q[j];
    const double T = two_theta_q(q, a.l2h, a.l2l, a.ttab);
    const double pos = (T - a.t0) * a.inv_dt;
    const double fb = floor(pos);
    float P = 1.f;
    if (c.po) {
        const uint32_t key = a.key[j];
        const float gn = fmaf((float)hkl_h(key), c.m0, fmaf((float)hkl_k(key), c.m1, (float)hkl_l(key) * c.m2));
        const float c2 = fminf(gn * gn / d2f_pos(q), 1.f);
        const float t = fmaf(c.r * c.r, c2, (1.f - c2) / c.r);
        P = 1.f / (t * sqrtf(t));
    }
    const float A = 2.f * a.Ig[j] * P;
    return make_float4(-(float)(int)fb, -(float)((pos - fb) * (double)c.sc), A * c.cl, A * c.cg);
}

// Lorentzian part of m staged reflections at a thread's kAugPts consecutive
// points (branch-free body; the unrolled iterations overlap). x at the thread's
// first point is exact up to rounding ((k - b) is an exact integer in FP32).
// EXACT computes every point the same way; otherwise x_j = x_0 + j s in one fma
// (absolute error a few ulp of kAugPts s: used for s <= 1, i.e. fwhm >= 2 dt).
template <bool EXACT>
__device__ __forceinline__ void aug_lorentz(const float4* __restrict__ st, int m, float kf, float sc,
                                            float (&acc)[kAugPts])
{
#pragma unroll 4
    for (int i = 0; i < m; i++) {
        const float4 R = st[i];  // (-b, -d s, Lorentzian amplitude, Gaussian amplitude)
        const float m0 = kf + R.x;
        float x[kAugPts];
#pragma unroll
        for (int j = 0; j < kAugPts; j++)
            x[j] = EXACT ? fmaf(m0 + (float)j, sc, R.y) : (j ? fmaf((float)j, sc, x[0]) : fmaf(m0, sc, R.y));
        // one reciprocal per pair of points: 1/d0 = d1 / (d0 d1). d <= 1 + 2^86 (2^23 grid
        // steps of at most 1e6 in x), so d0 d1 only overflows where both d exceed 2^42
        // (both terms below 2^-42 of the reflection's peak), and then both become 0.
#pragma unroll
        for (int j = 0; j < kAugPts; j += 2) {
            const float d0 = fmaf(x[j], x[j], 1.f), d1 = fmaf(x[j + 1], x[j + 1], 1.f);
            const float r = R.z * rcp_approx(d0 * d1);
            acc[j] = fmaf(d1, r, acc[j]);
            acc[j + 1] = fmaf(d0, r, acc[j + 1]);
        }
    }
}

// Gaussian part of the staged reflections that reach this warp's points (bit i
// of near[i / 32], set where |x| at the warp's centre is below half the warp's
// span in x plus sqrt(40)), in reflection order.
__device__ __forceinline__ void aug_gauss(const float4* __restrict__ st, const uint32_t* __restrict__ near, int m,
                                          float kf, float sc, float (&acc)[kAugPts])
{
    for (int w = 0; w < (m + 31) >> 5; w++) {
        uint32_t bits = near[w];
        while (bits) {
            const int i = 32 * w + __ffs(bits) - 1;
            bits &= bits - 1;
            const float4 R = st[i];
            const float m0 = kf + R.x;
#pragma unroll
            for (int j = 0; j < kAugPts; j++) {
                const float x = fmaf(m0 + (float)j, sc, R.y);
                acc[j] = fmaf(R.w, ex2_approx(-x * x), acc[j]);
            }
        }
    }
}

__global__ void __launch_bounds__(kAugThreads) k_aug_sum(const AugArgs a, int nblk)
{
    pdl_enter();
    __shared__ float4 st[kAugChunk];
    __shared__ uint32_t near[kAugWarps][kAugChunk / 32];  // reflections whose Gaussian reaches warp w
    __shared__ AugStruct cs;
    const int ib = blockIdx.x / nblk;
    const int s = a.aorder[ib];
    const int k0 = (blockIdx.x - ib * nblk) * kAugSpan;
    if (threadIdx.x == 0) {
        bool bad;
        cs = aug_struct(a, s, bad);
        if (bad && k0 == 0) {  // flagged once, by the structure's first CTA
            a.status[s] = XRD_EINVAL;
            atomicAdd((unsigned long long*)&a.totals[3], 1ull);
        }
    }
    __syncthreads();
    const AugStruct c = cs;
    const int kt = k0 + kAugPts * (int)threadIdx.x;  // this thread's first grid point
    const float kf = (float)kt;
    float acc[kAugPts];
#pragma unroll
    for (int j = 0; j < kAugPts; j++) acc[j] = 0.f;
    // warp w's points: k0 + 256 w .. k0 + 256 w + 255; none can reach x^2 < 40 when |x| at
    // their centre exceeds half their span in x plus sqrt(40) (with margin)
    const float kc0 = (float)k0 + 0.5f * (float)(32 * kAugPts - 1);
    const float reach = fmaf(0.5f * (float)(32 * kAugPts - 1), c.sc, 6.5f) * 1.0001f;
    const int warp = threadIdx.x >> 5;
    const int64_t base = c.n ? a.refl_off[s] : 0;
    for (int c0 = 0; c0 < c.n; c0 += kAugChunk) {
        const int m = min(kAugChunk, c.n - c0);
        __syncthreads();
        // whole warps stage 32 consecutive reflections each, so a ballot is one word of near[w]
        for (int i = threadIdx.x; i < ((m + 31) & ~31); i += kAugThreads) {
            float4 R = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < m) {
                R = aug_record(a, c, base + c0 + i);
                st[i] = R;
            }
#pragma unroll
            for (int w = 0; w < kAugWarps; w++) {
                const float kcw = kc0 + (float)(32 * kAugPts * w);
                const bool nr = i < m && c.gau && fabsf(fmaf(kcw + R.x, c.sc, R.y)) < reach;
                const uint32_t bal = __ballot_sync(0xffffffffu, nr);
                if ((threadIdx.x & 31) == 0) near[w][i >> 5] = bal;
            }
        }
        __syncthreads();
        if (c.lor) {
            if (c.sc <= 1.f) aug_lorentz<false>(st, m, kf, c.sc, acc);
            else aug_lorentz<true>(st, m, kf, c.sc, acc);
        }
        if (c.gau) aug_gauss(st, near[warp], m, kf, c.sc, acc);
    }
    const bool noise = c.valid && a.noise_z != nullptr;
    float* __restrict__ yo = a.y + (int64_t)s * a.n_pts;
    const float* __restrict__ zo = noise ? a.noise_z + (int64_t)s * a.n_pts : nullptr;
#pragma unroll
    for (int j = 0; j < kAugPts; j++) {
        const int k = kt + j;
        if (k >= a.n_pts) break;
        float v = acc[j];
        if (noise) v = fmaf(c.sig * sqrtf(fmaxf(v, 0.f)), zo[k], v);
        yo[k] = c.valid ? v : 0.f;
    }
}

void launch_aug(const AugArgs& a, cudaStream_t st)
{
    if (a.n_struct <= 0) return;
    const int nblk = (a.n_pts + kAugSpan - 1) / kAugSpan;
    launch_pdl(k_aug_order, 1, 1024, 0, st, a);
    launch_pdl(k_aug_sum, (unsigned)((int64_t)a.n_struct * nblk), kAugThreads, 0, st, a, nblk);
}

}  // namespace xrd
