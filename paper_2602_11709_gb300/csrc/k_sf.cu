// Steps S2-S3: per-reflection scalars, structure factor and intensity.
//
// Sec. 2: per reflection, the sum of the atoms' contributions (the structure
// factor), corrected by the Lorentz-polarisation and Debye-Waller factors:
//   F(g) = sum_j occ_j f_j(s) exp(-B_j s^2) exp(2 pi i (h x_j + k y_j + l z_j)),
//   f(s) = Z - 41.78214 s^2 sum_i a_i exp(-b_i s^2),  s = |g| / 2,
//   I = |F|^2 (1 + cos^2 2theta) / (sin^2 theta cos theta),  sin theta = lambda |g| / 2.
//
// GB300 mapping: every warp of a persistent grid takes 128-reflection tiles of
// one structure (four reflections per lane) from an atomic queue in
// largest-first order. The warp stages the structure's atoms in shared memory
// and every lane walks the same atom list (one broadcast read per atom feeds
// four terms). Atoms are sorted by
// element, so f(s) is evaluated once per element run (a warp-uniform branch).
// The pattern variants form sin/cos on the FMA pipe from the exact phase
// (sincos_turn32) and use the SFU for exp2 (MUFU.EX2); the gradient variant
// uses the SFU for sin/cos too (MUFU.SIN/COS). FP64 arithmetic runs at
// about 1/64 of the FP32 rate here, so the phase is reduced either in FP64
// (XRD_FP32_PHASE64) or exactly in 32-bit integers (XRD_FP32_PHASEFIX).
#include "xrd_internal.cuh"
#include "xrd_launch.h"

namespace xrd {

constexpr float kTwoPiOver2p32 = 1.4629180792671596e-09f;  // 2 pi / 2^32

// Launch shapes (chosen by xrd_autotune; default RB = 4, 2 warps per CTA):
// RB reflections per lane (one atom record feeds RB terms; tile = 32 RB
// reflections per warp) and WARPS warps per CTA.
constexpr int kSfChunk = 128;  // atoms staged per warp at a time

__device__ __forceinline__ float f_of(const Coef32& c, float zf, float s2)
{
    const float e0 = ex2_approx(c.bl[0] * s2), e1 = ex2_approx(c.bl[1] * s2);
    const float e2 = ex2_approx(c.bl[2] * s2), e3 = ex2_approx(c.bl[3] * s2);
    return fmaf(s2, fmaf(c.a[0], e0, fmaf(c.a[1], e1, fmaf(c.a[2], e2, c.a[3] * e3))), zf);
}

// Lorentz-polarisation factor (1 + cos^2 2theta) / (sin^2 theta cos theta) with
// sin^2 theta = X = q lambda^2 / 4. Up to 2theta = 90 degrees (X <= 1/2) the FP32
// cos^2 theta = 1 - X is good to a few ulp; above, its relative error grows as
// 1 / cos^2 theta (about 1.6e-5 at 170 degrees), so it is formed from |g|^2 in
// FP64 there (q: the reflection's |g|^2).
__device__ __forceinline__ float lp_of(float qf, float l2, const double* q, double lambda)
{
    const float X = qf * l2;  // sin^2 theta
    float u = 1.f - X;        // cos^2 theta
    if (X > 0.5f) u = fmaxf((float)fma(-0.25 * lambda * lambda, *q, 1.0), (float)kCos90Sq);
    const float c2 = fmaf(-2.f, X, 1.f);
    return fmaf(c2, c2, 1.f) / (X * sqrtf(u));
}

// d f / d s^2 = -41.78214 sum_i a_i exp(-b_i s^2)(1 - b_i s^2); with b_i = -bl_i ln 2
__device__ __forceinline__ float fprime_of(const Coef32& c, float s2)
{
    constexpr float ln2 = 0.69314718055994531f;
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < 4; i++) acc = fmaf(c.a[i] * ex2_approx(c.bl[i] * s2), fmaf(c.bl[i] * ln2, s2, 1.f), acc);
    return acc;
}

// The reflections of one lane in a tile: RUNS: one run of `len` reflections
// consecutive in l from `first` (step 1); otherwise up to RB reflections from
// `first` with a step of 32 (a tile of 32 RB consecutive reflections), `len` of
// them inside the structure.
//
// FP32 variants: every atom record (staged by the warp in shared memory, read
// by all lanes as a broadcast) feeds the lane's RB terms. With the integer phase
// (XRD_FP32_PHASEFIX) and RUNS, the phase factor is formed exactly once per run
// and atom, rotated from l to l + 1 by the atom's exp(2 pi i z) (an accurately
// rounded FP32 pair), and carried to l + 2 and l + 3 by the two-term recurrence
// e^{i(k+1)t} = 2 cos t e^{ikt} - e^{i(k-1)t} (two operations instead of four;
// rounding grows by a few ulp over a run of four): one sin/cos pair per run
// instead of per reflection. Otherwise every reflection's phase is formed exactly (integer
// phase) or in FP64 (XRD_FP32_PHASE64).
//
// Pattern variants (not GRAD): sin and cos come from the FMA pipe
// (sincos_turn32, five times more accurate than the SFU's), F is summed in FP32
// over blocks of 8 atoms (16 with runs) and
// each block sum is added into a two-float total (Knuth's TwoSum), so the
// rounding of the sum grows with the block size instead of the atom count
// (plain FP32 summation over N atoms errs by about 2e-8 sqrt(N) of the terms'
// root-sum-square). The lane also sums a_j^2, a_j = occ_j exp(-B_j s^2)
// max(|f_j|, Z_j), the scale of each term's rounding error (f_j itself may
// cancel to near zero; its rounding does not), and stores it for the
// re-evaluation of weak reflections (k_refine); with runs, once per run (its
// reflections, consecutive in l, have nearly equal s^2). Returns the lane's
// largest I.
// GRAD also accumulates dF/ds^2 = sum_j occ_j exp(-B_j s^2)(f_j' - B_j f_j) e^{i phi_j}.
template <int PREC, bool GRAD, int kSfRB, bool RUNS>
__device__ float sf_tile_fp32(const SfArgs& a, int s, int64_t first, int len, int64_t j0, int64_t j1, Atom32* sat,
                              float2* sstep, const Coef32* scoef, bool staged)
{
    constexpr float ln2 = 0.69314718055994531f;
    constexpr int step = RUNS ? 1 : 32;
    constexpr bool ACC = !GRAD;  // blocked two-float sum and the error scale
    const int lane = threadIdx.x & 31;
    float s2[kSfRB], Fr[kSfRB], Fi[kSfRB], f[kSfRB];
    float Gr[kSfRB], Gi[kSfRB], fp[kSfRB];
    float Rh[kSfRB], Rl[kSfRB], Ih[kSfRB], Il[kSfRB], A2[kSfRB];
    uint32_t uh[kSfRB], uk[kSfRB], ul[kSfRB];
#pragma unroll
    for (int i = 0; i < kSfRB; i++) {
        const int64_t r = first + (int64_t)step * (i < len ? i : 0);
        s2[i] = d2f_pos(a.q[r]) * 0.25f;
        if (!RUNS || i == 0) {
            const uint32_t key = a.key[r];
            uh[i] = (uint32_t)hkl_h(key); uk[i] = (uint32_t)hkl_k(key); ul[i] = (uint32_t)hkl_l(key);
        } else {
            uh[i] = uh[0]; uk[i] = uk[0]; ul[i] = ul[0] + (uint32_t)i;
        }
        Fr[i] = 0.f; Fi[i] = 0.f; f[i] = 0.f;
        Gr[i] = 0.f; Gi[i] = 0.f; fp[i] = 0.f;
        Rh[i] = 0.f; Rl[i] = 0.f; Ih[i] = 0.f; Il[i] = 0.f; A2[i] = 0.f;
    }
    constexpr bool kRotate = RUNS && PREC == XRD_FP32_PHASEFIX;
    constexpr int kFoldMask = kRotate ? 15 : 7;  // block size of the two-float sum: 16 atoms with runs, else 8
    int zc = -1;
    for (int64_t c0 = j0; c0 < j1; c0 += kSfChunk) {
        const int nc = (int)min((int64_t)kSfChunk, j1 - c0);
        if (!staged) {
            __syncwarp();
            for (int i = lane; i < nc; i += 32) {
                sat[i] = a.atom32[c0 + i];
                if (kRotate) sstep[i] = a.astep[c0 + i];
            }
            __syncwarp();
        }
        for (int jj = 0; jj < nc; jj++) {
            const Atom32 at = sat[jj];
            if (at.z != zc) {  // uniform: every lane walks the same element-sorted list
                zc = at.z;
                const Coef32 c = scoef[zc];
#pragma unroll
                for (int i = 0; i < kSfRB; i++) {
                    f[i] = f_of(c, at.zf, s2[i]);
                    if (GRAD) fp[i] = fprime_of(c, s2[i]);
                }
            }
            float cs = 0.f, sn = 0.f, cz = 1.f, sz = 0.f, tcz = 2.f, cp = 0.f, sp = 0.f;
            double dx = 0.0, dy = 0.0, dz = 0.0;
            if (kRotate) {
                const uint32_t P = uh[0] * at.X + uk[0] * at.Y + ul[0] * at.Z;
                if (ACC) sincos_turn32(P, sn, cs);
                else __sincosf((float)(int32_t)P * kTwoPiOver2p32, &sn, &cs);
                const float2 st = sstep[jj];
                cz = st.x;
                sz = st.y;
                tcz = cz + cz;  // exact
            } else if (PREC == XRD_FP32_PHASE64) {
                const Atom64 d = a.atom64[c0 + jj];
                dx = d.x; dy = d.y; dz = d.z;
            }
            const bool fold = ACC && ((jj & kFoldMask) == kFoldMask || jj == nc - 1);  // uniform
#pragma unroll
            for (int i = 0; i < kSfRB; i++) {
                if (!kRotate) {
                    uint32_t P;
                    if (PREC == XRD_FP32_PHASEFIX)
                        P = uh[i] * at.X + uk[i] * at.Y + ul[i] * at.Z;
                    else
                        P = fix32(fma((double)(int)uh[i], dx, fma((double)(int)uk[i], dy, (double)(int)ul[i] * dz)));
                    if (ACC) sincos_turn32(P, sn, cs);
                    else __sincosf((float)(int32_t)P * kTwoPiOver2p32, &sn, &cs);
                }
                const float dw = ex2_approx(fmaf(at.nb, s2[i], at.lo));
                const float w = f[i] * dw;
                Fr[i] = fmaf(w, cs, Fr[i]);
                Fi[i] = fmaf(w, sn, Fi[i]);
                if (ACC) {
                    if (!kRotate || i == 0) {  // a run's reflections share one scale (s^2 nearly equal)
                        const float m = dw * fmaxf(fabsf(f[i]), at.zf);
                        A2[i] = fmaf(m, m, A2[i]);
                    }
                    if (fold) {  // block sum into the two-float total
                        float t = Rh[i] + Fr[i], bb = t - Rh[i];
                        Rl[i] += (Rh[i] - (t - bb)) + (Fr[i] - bb);
                        Rh[i] = t;
                        t = Ih[i] + Fi[i];
                        bb = t - Ih[i];
                        Il[i] += (Ih[i] - (t - bb)) + (Fi[i] - bb);
                        Ih[i] = t;
                        Fr[i] = 0.f;
                        Fi[i] = 0.f;
                    }
                }
                if (GRAD) {
                    const float wd = fmaf(at.nb * ln2, f[i], fp[i]) * dw;
                    Gr[i] = fmaf(wd, cs, Gr[i]);
                    Gi[i] = fmaf(wd, sn, Gi[i]);
                }
                if (kRotate && i + 1 < kSfRB) {  // exp(2 pi i g.x) from l to l + 1
                    float c2, s2n;
                    if (i == 0) {  // the rotation by exp(2 pi i z)
                        c2 = fmaf(cs, cz, -sn * sz);
                        s2n = fmaf(cs, sz, sn * cz);
                    } else {  // two-term recurrence: e^{i(k+1)t} = 2 cos t e^{ikt} - e^{i(k-1)t}
                        c2 = fmaf(tcz, cs, -cp);
                        s2n = fmaf(tcz, sn, -sp);
                    }
                    cp = cs;
                    sp = sn;
                    cs = c2;
                    sn = s2n;
                }
            }
        }
    }
    const float l2 = (float)(a.lambda * a.lambda * 0.25);
    float imax = 0.f;
#pragma unroll
    for (int i = 0; i < kSfRB; i++) {
        if (i >= len) continue;
        const int64_t r = first + (int64_t)step * i;
        const float qf = d2f_pos(a.q[r]);
        const float fr = ACC ? Rh[i] + Rl[i] : Fr[i], fi = ACC ? Ih[i] + Il[i] : Fi[i];
        const float F2 = fmaf(fr, fr, fi * fi), lp = lp_of(qf, l2, a.q + r, a.lambda);
        const float I = F2 * lp;
        if (GRAD) {
            a.Fx[r] = make_float4(Fr[i], Fi[i], Gr[i], Gi[i]);
            a.Ig[r] = I;
        } else {
            a.If[r] = I;
            if (ACC && a.Eb) {
                // the bound of the rounding error of I; a reflection can need the re-evaluation only if
                // it exceeds tau of I (the criterion is E > tau max(I, c M)): then its structure is noted
                const float dF = a.eps_k * sqrtf(A2[kRotate ? 0 : i]);
                const float E = lp * dF * fmaf(2.f, sqrtf(F2), dF);
                a.Eb[r] = E;
                if (E > a.tau * I) a.Es[r] = s;
            }
            if (a.F) a.F[r] = make_float2(fr, fi);
            imax = fmaxf(imax, I);
        }
    }
    return imax;
}

// FP64 path: the lane's reflections one after another, every term in FP64.
template <int kSfRB>
__device__ void sf_tile_fp64(const SfArgs& a, int64_t first, int step, int len, int64_t j0, int64_t j1)
{
    for (int i = 0; i < kSfRB; i++) {
        const bool act = i < len;
        const int64_t r = first + (int64_t)step * (act ? i : 0);
        const double q = a.q[r];
        const uint32_t key = a.key[r];
        const int h = hkl_h(key), k = hkl_k(key), l = hkl_l(key);
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
        const double lp = (1.0 + c2 * c2) / (X * sqrt(fmax(1.0 - X, kCos90Sq)));
        if (act) {
            a.I[r] = (Fr * Fr + Fi * Fi) * lp;
            if (a.F) a.F[r] = make_float2((float)Fr, (float)Fi);
        }
    }
}

// Persistent CTAs; every warp takes tiles of 32 runs (one per lane) from a
// queue in largest-first order (tiles of the structures with the most atoms
// first). A structure's atoms stay staged in the warp's shared memory while its
// consecutive tiles follow (when they fit one chunk).
// Register caps: 64 for the integer-phase variant with 2 reflections per lane
// (32 resident warps per SM), about 85 for the other FP32 variants (24 warps).
template <int PREC, bool GRAD, int RB, int WARPS, bool RUNS>
__global__ void __launch_bounds__(32 * WARPS, PREC == XRD_FP64
                                                  ? 1
                                                  : ((PREC == XRD_FP32_PHASEFIX && !GRAD && RB == 2) ? 32 / WARPS
                                                                                                     : 24 / WARPS))
    k_sf(const SfArgs a)
{
    pdl_enter();
    constexpr int kSfThreads = 32 * WARPS;
    __shared__ Atom32 sat[WARPS][kSfChunk];
    __shared__ float2 sstep[WARPS][kSfChunk];
    extern __shared__ Coef32 scoef[];  // [zmax + 1]
    if (*a.abort_flag) return;
    const int ntiles = a.tile_off[a.n_struct];
    if (PREC != XRD_FP64) {
        for (int z = threadIdx.x; z <= a.zmax; z += kSfThreads) scoef[z] = a.coef32[z];
        __syncthreads();
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int staged_s = -1;  // structure whose atoms (one chunk at most) are in sat[w]
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.tile_counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        const int2 e = a.tile_tab[t];
        const int s = e.x;
        const int64_t rbase = a.refl_off[s], re = a.refl_off[s + 1];
        const int64_t j0 = a.atom_off[s], j1 = a.atom_off[s + 1];
        int64_t first;
        int len;
        if (RUNS) {  // lane: one run of the structure
            const int64_t nruns = a.run_cnt[s];
            const int64_t r = e.y + lane;
            int start = 0;
            len = 0;
            if (r < nruns) {
                const int pk = a.runs[rbase + r];
                start = pk >> 3;
                len = pk & 7;
            }
            first = rbase + start;
        } else {  // lane: reflections e.y + lane + 32 i of the structure
            first = rbase + e.y + lane;
            len = (int)max(min((re - first + 31) / 32, (int64_t)RB), (int64_t)0);
        }
        if (len == 0) first = rbase;  // keep the lane's (ignored) loads inside the array
        if (PREC == XRD_FP64) {
            sf_tile_fp64<RB>(a, first, RUNS ? 1 : 32, len, j0, j1);
        } else {
            const bool one_chunk = j1 - j0 <= kSfChunk;
            float m = sf_tile_fp32<PREC, GRAD, RB, RUNS>(a, s, first, len, j0, j1, sat[w], sstep[w], scoef,
                                                         one_chunk && s == staged_s);
            staged_s = one_chunk ? s : -1;
            if (!GRAD && a.imax) {  // the structure's largest reflection intensity (I >= 0: integer order)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0 && m > 0.f) atomicMax(a.imax + s, __float_as_uint(m));
            }
        }
    }
}

template <int PREC, bool GRAD, int RB, int WARPS, bool RUNS>
static void launch_sf_shape(const SfArgs& a, cudaStream_t st, bool pdl)
{
    // persistent grid: as many CTAs as fit on the SMs at once (cached per device and zmax)
    static int cache_per_sm[64] = {}, cache_zmax[64] = {};
    const size_t smem = PREC == XRD_FP64 ? 0 : sizeof(Coef32) * (size_t)(a.zmax + 1);
    int dev = 0;
    cudaGetDevice(&dev);
    const bool cached = dev >= 0 && dev < 64 && cache_per_sm[dev] > 0 && cache_zmax[dev] == a.zmax;
    int per_sm = cached ? cache_per_sm[dev] : 0;
    if (!cached) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sf<PREC, GRAD, RB, WARPS, RUNS>, 32 * WARPS,
                                                          smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 4;
        if (dev >= 0 && dev < 64) { cache_per_sm[dev] = per_sm; cache_zmax[dev] = a.zmax; }
    }
    if (pdl) launch_pdl(k_sf<PREC, GRAD, RB, WARPS, RUNS>, a.grid * per_sm, 32 * WARPS, smem, st, a);
    else k_sf<PREC, GRAD, RB, WARPS, RUNS><<<a.grid * per_sm, 32 * WARPS, smem, st>>>(a);
}

template <int PREC, bool GRAD>
static void launch_sf_prec(const SfArgs& a, cudaStream_t st, bool pdl)
{
    if (a.rb == 2) launch_sf_shape<PREC, GRAD, 2, 2, false>(a, st, pdl);
    else launch_sf_shape<PREC, GRAD, 4, 2, false>(a, st, pdl);
}

// a.grid = number of SMs; a.rb, a.warps, a.runs_mode = launch shape. Runs (with the l-step
// rotation) exist for the integer-phase pattern variant with 4 reflections per lane.
void launch_sf(const SfArgs& a, cudaStream_t st, bool pdl)
{
    if (a.n_struct <= 0) return;
    if (a.Fx) {  // gradient path: FP32 with the integer phase
        launch_sf_prec<XRD_FP32_PHASEFIX, true>(a, st, pdl);
        return;
    }
    switch (a.precision) {
    case XRD_FP64: launch_sf_prec<XRD_FP64, false>(a, st, pdl); break;
    case XRD_FP32_PHASE64: launch_sf_prec<XRD_FP32_PHASE64, false>(a, st, pdl); break;
    default:
        if (a.runs_mode) {
            if (a.warps == 1) launch_sf_shape<XRD_FP32_PHASEFIX, false, 4, 1, true>(a, st, pdl);
            else if (a.warps == 4) launch_sf_shape<XRD_FP32_PHASEFIX, false, 4, 4, true>(a, st, pdl);
            else launch_sf_shape<XRD_FP32_PHASEFIX, false, 4, 2, true>(a, st, pdl);
        } else if (a.rb == 2) {
            if (a.warps == 1) launch_sf_shape<XRD_FP32_PHASEFIX, false, 2, 1, false>(a, st, pdl);
            else if (a.warps == 4) launch_sf_shape<XRD_FP32_PHASEFIX, false, 2, 4, false>(a, st, pdl);
            else launch_sf_shape<XRD_FP32_PHASEFIX, false, 2, 2, false>(a, st, pdl);
        } else {
            if (a.warps == 1) launch_sf_shape<XRD_FP32_PHASEFIX, false, 4, 1, false>(a, st, pdl);
            else if (a.warps == 4) launch_sf_shape<XRD_FP32_PHASEFIX, false, 4, 4, false>(a, st, pdl);
            else launch_sf_shape<XRD_FP32_PHASEFIX, false, 4, 2, false>(a, st, pdl);
        }
        break;
    }
}

}  // namespace xrd
