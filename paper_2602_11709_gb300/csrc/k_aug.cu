// Augmented pattern: the experimental effects that synthetic training patterns
// for ML models carry (Sec. 1: peak broadening, noise, preferred orientation),
// applied on the GPU to the structure factors of the pattern path.
//
//   y_k = sum_g 2 I_g P_g PV(t_k - 2theta_g)   (Friedel-unique g; g and -g share I, P, 2theta)
//   P_g = (r^2 c + (1 - c) / r)^(-3/2),  c = cos^2 of the angle between g and n (metric G*)
//   PV(u) = eta (2 / (pi w)) / (1 + x^2) + (1 - eta) (2 / w) sqrt(ln 2 / pi) 2^(-x^2),  x = 2 u / w
//   then y_k += sigma sqrt(max(y_k, 0)) z_k.
//
// k_aug_refl (one CTA per structure) turns each reflection into a record: its
// grid cell b, the offset d of 2theta within the cell scaled by 2 dt / w, and the
// Lorentzian and Gaussian amplitudes. k_aug_sum gives each CTA 1024 grid points
// of one structure and streams all of the structure's reflections through
// shared memory: every (point, reflection) pair costs one reciprocal (MUFU) for
// the Lorentzian, which has no window; the Gaussian is evaluated only where a
// warp's 32 consecutive points reach x^2 < 40.
//
// Precision: x = (k - b) s - d s with k - b an exact integer in FP32 (|k|, |b| < 2^22),
// so x carries a relative error of a few ulp wherever it matters (|x| small);
// sums are FP32 in reflection order.
#include <cmath>

#include "xrd_internal.cuh"
#include "xrd_launch.h"

namespace xrd {

constexpr int kAugThreads = 256;
constexpr int kAugPts = 4;                       // grid points per thread (stride 256)
constexpr int kAugSpan = kAugThreads * kAugPts;  // grid points per CTA
constexpr int kAugChunk = 1024;                  // reflections staged in shared memory at a time
constexpr float kAugGaussX2 = 40.f;              // 2^-40: Gaussian skipped beyond on a whole warp
constexpr int kAugLor = 1, kAugGau = 2, kAugValid = 4;

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(kAugThreads) k_aug_refl(const AugArgs a)
{
    pdl_enter();
    const int s = blockIdx.x;
    const bool geo_ok = !*a.abort_flag && a.geo[s].status == XRD_OK;
    const double w = a.fwhm[s], eta = a.eta[s];
    const double sc = 2.0 * a.dt / w;
    // every comparison is false for NaN, so NaN parameters fail
    bool ok = w > 0.0 && w <= 1e6 && sc <= 1e6 && eta >= 0.0 && eta <= 1.0;
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, r = 1.f;
    const bool po = a.po_dir != nullptr;
    if (po && geo_ok) {
        // m = G* n / sqrt(n^T G* n): then g.n / |n| = h m0 + k m1 + l m2
        const double* n = a.po_dir + 3 * (int64_t)s;
        const double* g = a.geo[s].gs;
        const double R = a.po_r[s];
        const double M0 = g[0] * n[0] + g[3] * n[1] + g[4] * n[2];
        const double M1 = g[3] * n[0] + g[1] * n[1] + g[5] * n[2];
        const double M2 = g[4] * n[0] + g[5] * n[1] + g[2] * n[2];
        const double nn = n[0] * M0 + n[1] * M1 + n[2] * M2;
        ok = ok && R >= 1e-6 && R <= 1e6 && nn > 0.0 && nn < INFINITY && fabs(M0) < INFINITY &&
             fabs(M1) < INFINITY && fabs(M2) < INFINITY;
        if (ok) {
            const double inv = 1.0 / sqrt(nn);
            m0 = (float)(M0 * inv);
            m1 = (float)(M1 * inv);
            m2 = (float)(M2 * inv);
            r = (float)R;
        }
    }
    if (a.noise_z) {
        const double sig = a.noise_sigma[s];
        ok = ok && sig >= 0.0 && sig < INFINITY;
    }
    const bool valid = ok && geo_ok;
    const int64_t base = a.refl_off[s];
    const int n = valid ? (int)(a.refl_off[s + 1] - base) : 0;
    if (threadIdx.x == 0) {
        if (!ok && geo_ok) {
            a.status[s] = XRD_EINVAL;
            atomicAdd((unsigned long long*)&a.totals[3], 1ull);
        }
        const int flags = valid ? (kAugValid | (eta > 0.0 ? kAugLor : 0) | (eta < 1.0 ? kAugGau : 0)) : 0;
        a.rec[s] = make_int4(n, __float_as_int(valid ? (float)sc : 0.f), flags, 0);
    }
    if (n == 0) return;
    const float cl = (float)(eta * 2.0 / (kPi * w));
    const float cg = (float)((1.0 - eta) * (2.0 / w) * sqrt(log(2.0) / kPi));
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t j = base + i;
        const double q = a.q[j];
        const double T = two_theta_q(q, a.l2h, a.l2l, a.ttab);
        const double pos = (T - a.t0) / a.dt;
        const double fb = floor(pos);
        float P = 1.f;
        if (po) {
            const uint32_t key = a.key[j];
            const float gn = fmaf((float)hkl_h(key), m0, fmaf((float)hkl_k(key), m1, (float)hkl_l(key) * m2));
            const float c2 = fminf(gn * gn / (float)q, 1.f);
            const float t = fmaf(r * r, c2, (1.f - c2) / r);
            P = 1.f / (t * sqrtf(t));
        }
        const float A = 2.f * a.Ig[j] * P;
        a.rb[j] = (int)fb;
        a.rd[j] = (float)((pos - fb) * sc);
        a.aL[j] = A * cl;
        a.aG[j] = A * cg;
    }
}

__global__ void __launch_bounds__(kAugThreads) k_aug_sum(const AugArgs a, int nblk)
{
    pdl_enter();
    __shared__ float4 st[kAugChunk];  // (b, d s, Lorentzian amplitude, Gaussian amplitude)
    const int s = blockIdx.x / nblk;
    const int k0 = (blockIdx.x - s * nblk) * kAugSpan;
    const int4 rec = a.rec[s];
    const int n = rec.x;
    const float sc = __int_as_float(rec.y);
    const bool lor = (rec.z & kAugLor) != 0, gau = (rec.z & kAugGau) != 0;
    float kf[kAugPts], accL[kAugPts], accG[kAugPts];
#pragma unroll
    for (int j = 0; j < kAugPts; j++) {
        kf[j] = (float)(k0 + j * kAugThreads + (int)threadIdx.x);
        accL[j] = 0.f;
        accG[j] = 0.f;
    }
    // CTA-wide test: no point of this CTA can reach x^2 < 40 when |x| at the
    // CTA's centre exceeds half its span in x plus sqrt(40) (with margin)
    const float kc = (float)k0 + 0.5f * (float)(kAugSpan - 1);
    const float reach = fmaf(0.5f * (float)(kAugSpan - 1), sc, 6.5f) * 1.0001f;
    const int64_t base = n ? a.refl_off[s] : 0;
    for (int c0 = 0; c0 < n; c0 += kAugChunk) {
        const int m = min(kAugChunk, n - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += kAugThreads) {
            const int64_t j = base + c0 + i;
            st[i] = make_float4((float)a.rb[j], a.rd[j], a.aL[j], a.aG[j]);
        }
        __syncthreads();
        for (int i = 0; i < m; i++) {
            const float4 R = st[i];
            float x[kAugPts];
#pragma unroll
            for (int j = 0; j < kAugPts; j++) x[j] = fmaf(kf[j] - R.x, sc, -R.y);
            if (lor) {
#pragma unroll
                for (int j = 0; j < kAugPts; j++) accL[j] = fmaf(R.z, rcp_approx(fmaf(x[j], x[j], 1.f)), accL[j]);
            }
            if (gau && fabsf(fmaf(kc - R.x, sc, -R.y)) < reach) {  // uniform over the CTA
#pragma unroll
                for (int j = 0; j < kAugPts; j++) {
                    const float x2 = x[j] * x[j];
                    if (__any_sync(0xffffffffu, x2 < kAugGaussX2)) accG[j] = fmaf(R.w, ex2_approx(-x2), accG[j]);
                }
            }
        }
    }
    const bool valid = (rec.z & kAugValid) != 0;
    const bool noise = valid && a.noise_z != nullptr;
    const float sig = noise ? (float)a.noise_sigma[s] : 0.f;
    float* __restrict__ yo = a.y + (int64_t)s * a.n_pts;
#pragma unroll
    for (int j = 0; j < kAugPts; j++) {
        const int k = k0 + j * kAugThreads + (int)threadIdx.x;
        if (k >= a.n_pts) continue;
        float v = accL[j] + accG[j];
        if (noise) v = fmaf(sig * sqrtf(fmaxf(v, 0.f)), a.noise_z[(int64_t)s * a.n_pts + k], v);
        yo[k] = valid ? v : 0.f;
    }
}

void launch_aug(const AugArgs& a, cudaStream_t st)
{
    if (a.n_struct <= 0) return;
    const int nblk = (a.n_pts + kAugSpan - 1) / kAugSpan;
    launch_pdl(k_aug_refl, a.n_struct, kAugThreads, 0, st, a);
    launch_pdl(k_aug_sum, (unsigned)((int64_t)a.n_struct * nblk), kAugThreads, 0, st, a, nblk);
}

}  // namespace xrd
