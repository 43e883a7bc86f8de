// Steps S2-S3: per-reflection scalars, structure factor and intensity.
//
// Sec. 2 of the paper: "the nested loops for structure-factor evaluation by
// summing atomic contributions for each reflection" with the
// Lorentz-polarisation and Debye-Waller corrections:
//   F(g) = sum_j occ_j f_j(s) exp(-B_j s^2) exp(2 pi i (h x_j + k y_j + l z_j)),
//   f(s) = Z - 41.78214 s^2 sum_i a_i exp(-b_i s^2),  s = |g| / 2,
//   I = |F|^2 (1 + cos^2 2theta) / (sin^2 theta cos theta),  sin theta = lambda |g| / 2.
//
// GB300 mapping: one thread per reflection, a CTA per tile of reflections of
// one structure, tiles taken round-robin by a persistent grid. All lanes of a
// warp walk the same atom list (a broadcast load per atom). Atoms are sorted by
// element, so f(s) is evaluated once per element run (a warp-uniform branch).
// The FP32 variants use the SFU for sin/cos (MUFU.SIN/COS) and exp2 (MUFU.EX2,
// which this part issues at twice the sin/cos rate). FP64 arithmetic runs at
// about 1/64 of the FP32 rate here, so the phase is reduced either in FP64
// (XRD_FP32_PHASE64) or exactly in 32-bit integers (XRD_FP32_PHASEFIX).
#include "xrd_internal.cuh"
#include "xrd_launch.h"

namespace xrd {

constexpr float kTwoPiOver2p32 = 1.4629180792671596e-09f;  // 2 pi / 2^32

__device__ __forceinline__ int tile_struct(const int* __restrict__ tile_off, int n, int t)
{
    int lo = 0, hi = n;  // largest lo with tile_off[lo] <= t
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tile_off[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int PREC>
__global__ void __launch_bounds__(128) k_sf(const SfArgs a)
{
    if (*a.abort_flag) return;
    const int ntiles = a.tile_off[a.n_struct];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int s = tile_struct(a.tile_off, a.n_struct, t);
        const int64_t rb = a.refl_off[s], re = a.refl_off[s + 1];
        const int64_t r = rb + (int64_t)(t - a.tile_off[s]) * blockDim.x + threadIdx.x;
        const bool act = r < re;
        const int64_t rr = act ? r : rb;
        const double q = a.q[rr];
        const uint32_t key = a.key[rr];
        const int h = hkl_h(key), k = hkl_k(key), l = hkl_l(key);
        const int64_t j0 = a.atom_off[s], j1 = a.atom_off[s + 1];
        double I;
        if (PREC == XRD_FP64) {
            const double s2 = q * 0.25;
            double Fr = 0.0, Fi = 0.0, f = 0.0;
            int zc = -1;
            for (int64_t j = j0; j < j1; j++) {
                const Atom64 at = a.atom64[j];
                if (at.zz != zc) {
                    zc = at.zz;
                    const double* c = a.coef + 8 * zc;
                    const double sum = c[0] * exp(-c[1] * s2) + c[2] * exp(-c[3] * s2) + c[4] * exp(-c[5] * s2) +
                                       c[6] * exp(-c[7] * s2);
                    f = (double)zc - kFScale * s2 * sum;
                }
                double phi = fma((double)h, at.x, fma((double)k, at.y, (double)l * at.z));
                phi -= rint(phi);
                double sn, cs;
                sincospi(2.0 * phi, &sn, &cs);
                const double w = at.occ * f * exp(-at.B * s2);
                Fr = fma(w, cs, Fr);
                Fi = fma(w, sn, Fi);
            }
            const double X = (a.lambda * a.lambda * 0.25) * q;  // sin^2 theta
            const double c2 = 1.0 - 2.0 * X;                     // cos 2theta
            const double lp = (1.0 + c2 * c2) / (X * sqrt(1.0 - X));
            I = (Fr * Fr + Fi * Fi) * lp;
            if (a.F && act) a.F[r] = make_float2((float)Fr, (float)Fi);
        } else {
            const float qf = d2f_pos(q);
            const float s2 = qf * 0.25f;
            const uint32_t uh = (uint32_t)h, uk = (uint32_t)k, ul = (uint32_t)l;
            float Fr = 0.f, Fi = 0.f, f = 0.f;
            int zc = -1;
            for (int64_t j = j0; j < j1; j++) {
                const Atom32 at = a.atom32[j];
                if (at.z != zc) {
                    zc = at.z;
                    const Coef32 c = a.coef32[zc];
                    const float e0 = ex2_approx(c.bl[0] * s2), e1 = ex2_approx(c.bl[1] * s2);
                    const float e2 = ex2_approx(c.bl[2] * s2), e3 = ex2_approx(c.bl[3] * s2);
                    f = fmaf(s2, fmaf(c.a[0], e0, fmaf(c.a[1], e1, fmaf(c.a[2], e2, c.a[3] * e3))), (float)zc);
                }
                uint32_t P;
                if (PREC == XRD_FP32_PHASEFIX) {
                    P = uh * at.X + uk * at.Y + ul * at.Z;
                } else {
                    const Atom64 d = a.atom64[j];
                    P = fix32(fma((double)h, d.x, fma((double)k, d.y, (double)l * d.z)));
                }
                float sn, cs;
                __sincosf((float)(int32_t)P * kTwoPiOver2p32, &sn, &cs);
                const float w = f * ex2_approx(fmaf(at.nb, s2, at.lo));
                Fr = fmaf(w, cs, Fr);
                Fi = fmaf(w, sn, Fi);
            }
            const float X = qf * (float)(a.lambda * a.lambda * 0.25);
            const float c2 = fmaf(-2.f, X, 1.f);
            const float lp = fmaf(c2, c2, 1.f) / (X * sqrtf(1.f - X));
            I = f2d_fast((Fr * Fr + Fi * Fi) * lp);
            if (a.F && act) a.F[r] = make_float2(Fr, Fi);
        }
        if (act) a.I[r] = I;
    }
}

void launch_sf(const SfArgs& a, cudaStream_t st)
{
    if (a.n_struct <= 0) return;
    switch (a.precision) {
    case XRD_FP64: k_sf<XRD_FP64><<<a.grid, 128, 0, st>>>(a); break;
    case XRD_FP32_PHASE64: k_sf<XRD_FP32_PHASE64><<<a.grid, 128, 0, st>>>(a); break;
    default: k_sf<XRD_FP32_PHASEFIX><<<a.grid, 128, 0, st>>>(a); break;
    }
}

}  // namespace xrd
