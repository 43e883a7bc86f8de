// Steps S0-S1: per-structure geometry, atom packing and reflection enumeration.
//
// Sec. 2: the first step of the numerical core enumerates the reciprocal-lattice
// points that the wavelength and the 2-theta range can reach (a sphere in
// reciprocal space): every integer g = (h, k, l) != 0 with r_min <= |g| <= r_max, |g|^2 = h^T G* h.
// Friedel's law F(-g) = F(g)* makes g and -g identical in intensity, so only
// the half-space (first nonzero of h, k, l positive) is enumerated; every kept
// reflection stands for two.
//
// |g|^2 is evaluated in one fixed order with every product and sum rounded on
// its own (no fused multiply-add), so the set of reflections on the sphere
// boundary is decided exactly as a plain FP64 evaluation of the same order.
#include "xrd_dd.cuh"
#include "xrd_internal.cuh"
#include "xrd_launch.h"

namespace xrd {

__device__ __forceinline__ double cosd(double deg)
{
    // exact cosines at 90, 60 and 120 degrees; otherwise cos(deg * pi / 180)
    if (deg == 90.0) return 0.0;
    if (deg == 60.0) return 0.5;
    if (deg == 120.0) return -0.5;
    return cos(__dmul_rn(deg, kPi / 180.0));
}

// S0: reciprocal metric G* = G^-1 from the direct metric
// G = [[a^2, ab cos(gamma), ac cos(beta)], [., b^2, bc cos(alpha)], [., ., c^2]]
// by cofactors over the determinant, and the enumeration box |h| <= r_max a + 1.
// The part has little FP64 throughput. A small batch is latency-bound, so
// each structure takes LANES = 8 lanes: lanes 0-2 form the three cosines,
// every lane the cofactors and determinant (same operations, same order), lane
// j < 6 the element j of G* (one division each), lane 6 the box, status and
// hexagonal flag. A large batch is throughput-bound and takes one lane per
// structure (LANES = 1, no redundant work). Every value is rounded exactly as
// in a one-thread evaluation either way.
// Also zeroes the structure's largest-intensity slot (imax, written by the
// structure-factor pass) and writes its flag word (bit 0: hexagonal) when the
// pointers are given.
template <int LANES>
__global__ void k_prep(const double* __restrict__ lattice, int n, double rmax, Geo* __restrict__ geo,
                       unsigned* __restrict__ imax, int32_t* __restrict__ flags)
{
    pdl_enter();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int s_raw = t / LANES, lane = t % LANES;
    const bool live = s_raw < n;
    if (LANES == 1 && !live) return;
    const int s = live ? s_raw : n - 1;  // lanes past the batch compute a copy and store nothing
    const double a = lattice[6 * s], b = lattice[6 * s + 1], c = lattice[6 * s + 2];
    const double al = lattice[6 * s + 3], be = lattice[6 * s + 4], ga = lattice[6 * s + 5];
    Geo& g = geo[s];
    const bool finite = isfinite(a) && isfinite(b) && isfinite(c) && isfinite(al) && isfinite(be) && isfinite(ga);
    bool ok = finite && a > 0.0 && b > 0.0 && c > 0.0;
    double ca, cb, cg;
    if (LANES == 1) {
        ca = ok ? cosd(al) : 0.0;
        cb = ok ? cosd(be) : 0.0;
        cg = ok ? cosd(ga) : 0.0;
    } else {
        const double cj = (ok && lane < 3) ? cosd(lane == 0 ? al : (lane == 1 ? be : ga)) : 0.0;
        ca = __shfl_sync(0xffffffffu, cj, 0, LANES);
        cb = __shfl_sync(0xffffffffu, cj, 1, LANES);
        cg = __shfl_sync(0xffffffffu, cj, 2, LANES);
    }
    // volume factor 1 - ca^2 - cb^2 - cg^2 + 2 ca cb cg, left to right
    double vf = __dsub_rn(1.0, __dmul_rn(ca, ca));
    vf = __dsub_rn(vf, __dmul_rn(cb, cb));
    vf = __dsub_rn(vf, __dmul_rn(cg, cg));
    vf = __dadd_rn(vf, __dmul_rn(__dmul_rn(__dmul_rn(2.0, ca), cb), cg));
    ok = ok && vf > 1e-6;
    const double G11 = __dmul_rn(a, a), G22 = __dmul_rn(b, b), G33 = __dmul_rn(c, c);
    const double G12 = __dmul_rn(__dmul_rn(a, b), cg);
    const double G13 = __dmul_rn(__dmul_rn(a, c), cb);
    const double G23 = __dmul_rn(__dmul_rn(b, c), ca);
    const double C11 = __dsub_rn(__dmul_rn(G22, G33), __dmul_rn(G23, G23));
    const double C12 = __dsub_rn(__dmul_rn(G13, G23), __dmul_rn(G12, G33));
    const double C13 = __dsub_rn(__dmul_rn(G12, G23), __dmul_rn(G13, G22));
    const double det = __dadd_rn(__dadd_rn(__dmul_rn(G11, C11), __dmul_rn(G12, C12)), __dmul_rn(G13, C13));
    if (!live) return;
#pragma unroll
    for (int j = (LANES == 1 ? 0 : lane); j < (LANES == 1 ? 7 : lane + 1); j++) {
        if (j < 6) {
            // element j of G* (stored as 11, 22, 33, 12, 13, 23)
            double Cj;
            switch (j) {
            case 0: Cj = C11; break;
            case 1: Cj = __dsub_rn(__dmul_rn(G11, G33), __dmul_rn(G13, G13)); break;
            case 2: Cj = __dsub_rn(__dmul_rn(G11, G22), __dmul_rn(G12, G12)); break;
            case 3: Cj = C12; break;
            case 4: Cj = C13; break;
            default: Cj = __dsub_rn(__dmul_rn(G12, G13), __dmul_rn(G11, G23)); break;
            }
            const double v = ok ? __ddiv_rn(Cj, det) : 0.0;
            g.gs[j] = v;
            if (j >= 3) g.g2[j - 3] = 2.0 * v;  // exact
            const float v32 = ok ? __double2float_rn(v) : 0.f;
            g.gf[j] = v32;
            g.gl[j] = ok ? __double2float_rn(v - (double)v32) : 0.f;
        } else if (j == 6) {
            g.hex = fabs(al - 90.0) < 5.0 && fabs(be - 90.0) < 5.0 && fabs(ga - 120.0) < 5.0 && fabs(a - b) < 0.01;
            if (imax) imax[s] = 0u;
            if (flags) flags[s] = g.hex ? XRD_FLAG_HEXAGONAL : 0;
            int H = -1, K = -1, L = -1, st = XRD_EINVAL;
            if (ok) {
                H = (int)floor(__dmul_rn(rmax, a)) + 1;
                K = (int)floor(__dmul_rn(rmax, b)) + 1;
                L = (int)floor(__dmul_rn(rmax, c)) + 1;
                st = XRD_OK;
                if (H > kHklLimit || K > kHklLimit || L > kHklLimit) {
                    st = XRD_EINVAL;  // cell too large for the packed (h, k, l) key at this 2-theta range
                    H = K = L = -1;
                }
            }
            g.H = H;
            g.K = K;
            g.L = L;
            g.status = st;
        }
    }
}

// 8 lanes per structure up to this many structures (latency-bound), one above (throughput-bound)
constexpr int kPrepWideMax = 8192;

static void prep_launch(bool pdl, const double* lattice, int n, double rmax, Geo* geo, unsigned* imax,
                        int32_t* flags, cudaStream_t st);

// f(s) coefficients in the form the FP32 loops use (exp2 with the scale folded
// in) and, for the accurate re-evaluation, (a_i, b_i) as two floats each
// (cdd[4 z + i] = (a hi, a lo, b hi, b lo); skipped when cdd is null).
__global__ void k_coef(const double* __restrict__ coef, int zmax, Coef32* __restrict__ c32, float4* __restrict__ cdd)
{
    pdl_enter();
    for (int z = threadIdx.x; z <= zmax; z += blockDim.x) {
        Coef32 c;
        for (int i = 0; i < 4; i++) {
            const double av = coef[8 * z + 2 * i], bv = coef[8 * z + 2 * i + 1];
            c.a[i] = (float)(-kFScale * av);
            c.bl[i] = (float)(-bv * 1.4426950408889634);
            if (cdd) {
                const float ah = __double2float_rn(av), bh = __double2float_rn(bv);
                cdd[4 * z + i] = make_float4(ah, __double2float_rn(av - (double)ah), bh,
                                             __double2float_rn(bv - (double)bh));
            }
        }
        c32[z] = c;
    }
}

// Validate and pack the atoms of one structure, sorted by element (stable:
// ties keep their input order) so that f(s) is evaluated once per element run.
__global__ void __launch_bounds__(128) k_atoms(const int64_t* __restrict__ atom_off, int64_t n_atoms,
                                               const double* __restrict__ frac, const int16_t* __restrict__ Zin,
                                               const double* __restrict__ occ, const double* __restrict__ Bf, int zmax,
                                               Geo* __restrict__ geo, int set_geo, int* __restrict__ atom_bad,
                                               Atom32* __restrict__ a32, Atom64* __restrict__ a64,
                                               float2* __restrict__ astep, AtomR* __restrict__ ar,
                                               const float4* __restrict__ sctab)
{
    pdl_enter();
    __shared__ int off[kZmaxLimit + 1];
    __shared__ int zs[128];
    __shared__ int bad;
    const int s = blockIdx.x;
    int64_t a0 = atom_off[s], na = atom_off[s + 1] - a0;
    const bool range_ok = a0 >= 0 && na >= 0 && atom_off[s + 1] <= n_atoms && na <= (1 << 30);
    if (!range_ok) { a0 = 0; na = 0; }
    for (int i = threadIdx.x; i <= kZmaxLimit; i += blockDim.x) off[i] = 0;
    if (threadIdx.x == 0) bad = !range_ok;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < na; i += blockDim.x) {
        const int z = Zin[a0 + i];
        const double x = frac[3 * (a0 + i)], y = frac[3 * (a0 + i) + 1], w = frac[3 * (a0 + i) + 2];
        const bool ok = z >= 0 && z <= zmax && isfinite(x) && isfinite(y) && isfinite(w) && occ[a0 + i] >= 0.0 &&
                        isfinite(occ[a0 + i]) &&
                        isfinite(Bf[a0 + i]) && fabs(x) < 262144.0 && fabs(y) < 262144.0 && fabs(w) < 262144.0;
        if (!ok) atomicOr(&bad, 1);
        else atomicAdd(&off[z], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) atom_bad[s] = bad;
    if (bad) {
        // neutral records (weight 0, element 0) keep the structure-factor kernel's reads in bounds;
        // the structure reports XRD_EINVAL and gets no peaks
        if (threadIdx.x == 0 && set_geo) geo[s].status = XRD_EINVAL;
        for (int64_t i = threadIdx.x; i < na; i += blockDim.x) {
            Atom32 r{};
            r.lo = -INFINITY;
            r.src = (int)i;
            a32[a0 + i] = r;
            Atom64 d{};
            a64[a0 + i] = d;
            if (astep) astep[a0 + i] = make_float2(1.f, 0.f);
            if (ar) {
                AtomR e{};
                ar[a0 + i] = e;
            }
        }
        return;
    }
    if (threadIdx.x < 32) {  // exclusive offset of each element's run: one warp, 8 elements a lane
        constexpr int per = (kZmaxLimit + 1) / 32;
        const int lane = threadIdx.x;
        int v[per], sum = 0;
#pragma unroll
        for (int k = 0; k < per; k++) {
            const int z = lane * per + k;
            v[k] = z <= zmax ? off[z] : 0;
            sum += v[k];
        }
        int run = warp_incl_scan(sum) - sum;
#pragma unroll
        for (int k = 0; k < per; k++) {
            const int z = lane * per + k;
            if (z <= zmax) off[z] = run;
            run += v[k];
        }
    }
    __syncthreads();
    // stable placement, one chunk of blockDim atoms at a time
    for (int64_t base = 0; base < na; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int z = i < na ? (int)Zin[a0 + i] : -1;
        zs[threadIdx.x] = z;
        __syncthreads();
        if (i < na) {
            int before = 0;
            for (int t = 0; t < (int)threadIdx.x; t++) before += zs[t] == z;
            const int pos = off[z] + before;
            const double x = frac[3 * (a0 + i)], y = frac[3 * (a0 + i) + 1], w = frac[3 * (a0 + i) + 2];
            const double o = occ[a0 + i], bb = Bf[a0 + i];
            Atom32 r;
            r.X = fix32(x);
            r.Y = fix32(y);
            r.Z = fix32(w);
            r.nb = (float)(-bb * 1.4426950408889634);
            r.lo = o == 1.0 ? 0.f : (o > 0.0 ? (float)log2(o) : -INFINITY);
            r.z = z;
            r.src = (int)i;
            r.zf = (float)z;
            a32[a0 + pos] = r;
            if (astep) {  // the l -> l + 1 step of the phase factor (runs), from the same fixed-point z:
                          // cos and sin of 2 pi z in double-float (FP32 operations), rounded to floats
                DD cz, sz;
                dd_sincos_turn((unsigned long long)r.Z << 32, sctab, cz, sz);
                astep[a0 + pos] = make_float2(cz.hi + cz.lo, sz.hi + sz.lo);
            }
            Atom64 d;
            d.x = x; d.y = y; d.z = w; d.B = bb; d.occ = o; d.zz = z; d.pad = 0;
            a64[a0 + pos] = d;
            if (ar) {  // the accurate re-evaluation's record: 64-bit fixed point, two-float occ and B
                AtomR e;
                e.X = fix64(x);
                e.Y = fix64(y);
                e.Z = fix64(w);
                e.oh = __double2float_rn(o);
                e.ol = __double2float_rn(o - (double)e.oh);
                e.bh = __double2float_rn(bb);
                e.bl = __double2float_rn(bb - (double)e.bh);
                e.z = z;
                e.pad = 0;
                ar[a0 + pos] = e;
            }
        }
        __syncthreads();  // every read of off[] for this chunk is done
        if (i < na) atomicAdd(&off[z], 1);
        __syncthreads();
    }
}

// |g|^2 in the fixed order ((G11 hh + G22 kk) + G33 ll) + 2 ((G12 hk + G13 hl) + G23 kl).
__device__ __forceinline__ double q_exact(const double* gs, int h, int k, int l)
{
    const double hh = (double)(h * h), kk = (double)(k * k), ll = (double)(l * l);
    const double hk = (double)(h * k), hl = (double)(h * l), kl = (double)(k * l);
    const double diag = __dadd_rn(__dadd_rn(__dmul_rn(gs[0], hh), __dmul_rn(gs[1], kk)), __dmul_rn(gs[2], ll));
    const double off = __dadd_rn(__dadd_rn(__dmul_rn(gs[3], hk), __dmul_rn(gs[4], hl)), __dmul_rn(gs[5], kl));
    return __dadd_rn(diag, __dmul_rn(2.0, off));
}

// The l interval of column (h, k) that can hold |g|^2 <= r2max, computed in
// FP32 and widened by two on each side (a superset: every l in it is tested).
__device__ __forceinline__ void column_range(const float* gf, int L, int h, int k, float r2maxf, int& lo, int& hi)
{
    const float fh = (float)h, fk = (float)k;
    const float A = fmaf(gf[0] * fh, fh, fmaf(gf[1] * fk, fk, 2.f * gf[3] * fh * fk));
    const float b = fmaf(gf[4], fh, gf[5] * fk);
    const float R = r2maxf * 1.0001f;
    const float c = A - R;
    float disc = fmaf(b, b, -gf[2] * c);
    const float mag = fmaf(b, b, gf[2] * fabsf(c));
    lo = 1;
    hi = 0;
    if (disc < -1e-4f * mag) return;
    disc = fmaxf(disc, 0.f);
    const float sq = sqrtf(disc);
    const float inv = 1.f / gf[2];
    lo = (int)floorf((-b - sq) * inv) - 2;
    hi = (int)ceilf((-b + sq) * inv) + 2;
    if (lo < -L) lo = -L;
    if (hi > L) hi = L;
    if (h == 0 && k == 0 && lo < 1) lo = 1;  // half-space: (0, 0, l > 0)
}

__device__ __noinline__ int q_side_exact(const double* gs, int h, int k, int l, double r);

// Side of |g|^2 against a squared radius r for one (h, k, l): an FP32
// evaluation decides every candidate farther from r than a bound on its
// rounding error; the rest compare the fixed-order FP64 value (q_exact).
// Returns -1 (|g|^2 < r), 0 (equal) or 1 (|g|^2 > r).
__device__ __forceinline__ int q_side(const Geo& g, const double* gsg, int h, int k, int l, double r, float rf)
{
    const float* gf = g.gf;
    const float hh = (float)(h * h), kk = (float)(k * k), ll = (float)(l * l);
    const float hk = (float)(h * k), hl = (float)(h * l), kl = (float)(k * l);
    const float diag = fmaf(gf[2], ll, fmaf(gf[1], kk, gf[0] * hh));
    const float o1 = gf[3] * hk, o2 = gf[4] * hl, o3 = gf[5] * kl;
    const float qf = fmaf(2.f, o1 + o2 + o3, diag);
    const float qa = fmaf(2.f, fabsf(o1) + fabsf(o2) + fabsf(o3), diag);
    const float m = 4e-6f * qa + 1e-30f;
    if (qf > rf + m) return 1;
    if (qf < rf - m) return -1;
    return q_side_exact(gsg, h, k, l, r);
}

// The reflections of column (h, k) are the l of [a, b] outside [c, d] (c > d:
// the column misses the inner sphere). Along a column |g|^2 is a convex
// quadratic in l; its second difference 2 G*33 exceeds the rounding error of the
// fixed-order FP64 value by many orders of magnitude, so the l that pass the
// per-reflection test r2min <= |g|^2 <= r2max are exactly an interval minus an
// inner interval. Their ends are found by testing l inward from the FP32
// superset bounds of column_range, a few tests per column instead of one per l.
struct ColSpan {
    int a, b, c, d;
    __device__ int count() const { return a > b ? 0 : (b - a + 1) - (c <= d ? d - c + 1 : 0); }
    __device__ int first_part() const { return a > b ? 0 : (c <= d ? c - a : b - a + 1); }  // l in [a, c)
};

__device__ __forceinline__ ColSpan column_span(const Geo& g, const double* gsg, int h, int k, double r2min,
                                               double r2max, float r2minf, float r2maxf)
{
    ColSpan sp{1, 0, 1, 0};
    int lo, hi;
    column_range(g.gf, g.L, h, k, r2maxf, lo, hi);
    while (lo <= hi && q_side(g, gsg, h, k, lo, r2max, r2maxf) > 0) lo++;
    while (hi > lo && q_side(g, gsg, h, k, hi, r2max, r2maxf) > 0) hi--;
    if (lo > hi) return sp;
    sp.a = lo;
    sp.b = hi;
    if (r2min > 0.0) {
        int c0, d0;
        column_range(g.gf, g.L, h, k, r2minf, c0, d0);
        c0 = max(c0, lo);
        d0 = min(d0, hi);
        while (c0 <= d0 && q_side(g, gsg, h, k, c0, r2min, r2minf) >= 0) c0++;
        while (d0 > c0 && q_side(g, gsg, h, k, d0, r2min, r2minf) >= 0) d0--;
        if (c0 <= d0) {
            sp.c = c0;
            sp.d = d0;
        }
    }
    return sp;
}

// Columns of the half-space (h > 0, or h = 0 and k >= 0) in their emission
// order: h ascending, then k ascending; l ascending within a column.
__device__ __forceinline__ int n_columns(const Geo& g)
{
    return (g.status == XRD_OK && g.H >= 0) ? (g.K + 1) + g.H * (2 * g.K + 1) : 0;
}
__device__ __forceinline__ void column_hk(const Geo& g, int c, int& h, int& k)
{
    if (c <= g.K) {
        h = 0;
        k = c;
        return;
    }
    const int nk = 2 * g.K + 1, r = c - (g.K + 1);
    h = 1 + r / nk;
    k = r % nk - g.K;
}

// Runs: the structure-factor kernel gives each lane a run of at most rb
// reflections that are consecutive in l within one column, so that it can step
// the phase factor exp(2 pi i g.x) from l to l + 1 by one complex rotation.
// Each of a column's (at most two) contiguous parts is cut into runs of rb
// from its first l, the last one shorter. Run entries: (first reflection
// within the structure) << 3 | length.
__device__ __forceinline__ int runs_of(int n, int rb) { return (n + rb - 1) / rb; }

// Exclusive block scan of one (x, y) pair per thread, with the block totals.
// tmp: 66 ints of shared memory; the caller synchronises before reusing it.
__device__ __forceinline__ void block_scan_pair(int x, int y, int* tmp, int& ex, int& ey, int& tx, int& ty)
{
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ix = warp_incl_scan(x), iy = warp_incl_scan(y);
    if (lane == 31) {
        tmp[w] = ix;
        tmp[33 + w] = iy;
    }
    __syncthreads();
    if (w == 0) {
        const int sx = lane < nw ? tmp[lane] : 0, sy = lane < nw ? tmp[33 + lane] : 0;
        const int px = warp_incl_scan(sx), py = warp_incl_scan(sy);
        if (lane < nw) {
            tmp[lane] = px - sx;
            tmp[33 + lane] = py - sy;
        }
        if (lane == 31) {
            tmp[32] = px;
            tmp[65] = py;
        }
    }
    __syncthreads();
    ex = tmp[w] + ix - x;
    ey = tmp[33 + w] + iy - y;
    tx = tmp[32];
    ty = tmp[65];
}

// Launch shapes of counting and emission (enum_threads): with 64, 128 or 256
// threads per CTA every warp takes one structure at a time, claimed from a
// counter, so the fixed cost of a structure (the loads of its cell, the
// scans) is a warp's, not a CTA's, and a small structure's columns fill a
// warp's lanes; with 512 or 1024 threads every structure has a CTA of its own
// (batches of large cells).
constexpr int kEnumMaxThreads = 1024;
constexpr int kWarpModeMaxThreads = 256;
constexpr int kWarpRecInts = 2 * 33 + 8 * 32;  // one warp's chunk of 32 column records

__host__ __device__ inline bool enum_per_warp(int threads) { return threads <= kWarpModeMaxThreads; }
__host__ __device__ inline int enum_cta_ints(int threads) { return 2 * (threads + 1) + 8 * threads; }
size_t enum_smem_bytes(int threads)
{
    return 4 * ((enum_per_warp(threads) ? (threads / 32) * kWarpRecInts : 0) + enum_cta_ints(threads));
}

// The exact comparison of a candidate within the FP32 error bound of a sphere
// surface, kept out of line so that the rare FP64 evaluation is a branch, not
// work that every caller does.
__device__ __noinline__ int q_side_exact(const double* gs, int h, int k, int l, double r)
{
    const double q = q_exact(gs, h, k, l);
    return q > r ? 1 : (q < r ? -1 : 0);
}

// Reflections and runs of column c.
__device__ __forceinline__ ColSpan column_counts(const Geo& g, const double* gsg, int c, double r2min, double r2max,
                                                 float r2minf, float r2maxf, int rb, bool runs, int& h, int& k, int& n,
                                                 int& nr)
{
    column_hk(g, c, h, k);
    const ColSpan sp = column_span(g, gsg, h, k, r2min, r2max, r2minf, r2maxf);
    n = sp.count();
    nr = 0;
    if (runs) {
        const int n1 = sp.first_part();
        nr = runs_of(n1, rb) + runs_of(n - n1, rb);
    }
    return sp;
}

__device__ __forceinline__ int warp_sum_int(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reflection (and, with rb > 0, run) counts per structure. With one warp per
// structure the warps claim structures from a counter (ctr, zero at launch),
// so a CTA is not held by its slowest structure; every structure, however
// many columns it has, is counted by one warp.
template <bool RUNS>
__global__ void __launch_bounds__(kEnumMaxThreads) k_count(const Geo* __restrict__ geo, int n_struct, double r2min,
                                                           double r2max, float r2minf, float r2maxf, int rb,
                                                           int64_t* __restrict__ cnt, int64_t* __restrict__ run_cnt,
                                                           int* __restrict__ ctr)
{
    pdl_enter();
    __shared__ int tmp[66];
    const int nt = blockDim.x, lane = threadIdx.x & 31;
    if (enum_per_warp(nt)) {
        for (;;) {
            int s = 0;
            if (lane == 0) s = atomicAdd(ctr, 1);
            s = __shfl_sync(0xffffffffu, s, 0);
            if (s >= n_struct) break;
            const Geo g = geo[s];
            const int ncol = n_columns(g);
            int local = 0, local_runs = 0;
            for (int c = lane; c < ncol; c += 32) {
                int h, k, m, mr;
                column_counts(g, geo[s].gs, c, r2min, r2max, r2minf, r2maxf, rb, RUNS, h, k, m, mr);
                local += m;
                local_runs += mr;
            }
            local = warp_sum_int(local);
            if (RUNS) local_runs = warp_sum_int(local_runs);
            if (lane == 0) {
                cnt[s] = local;
                if (RUNS && run_cnt) run_cnt[s] = local_runs;
            }
        }
        return;
    }
    const int sb = blockIdx.x;  // one CTA per structure
    if (sb >= n_struct) return;
    const Geo g = geo[sb];
    const int ncol = n_columns(g);
    int local = 0, local_runs = 0;
    for (int c = threadIdx.x; c < ncol; c += nt) {
        int h, k, m, mr;
        column_counts(g, geo[sb].gs, c, r2min, r2max, r2minf, r2maxf, rb, RUNS, h, k, m, mr);
        local += m;
        local_runs += mr;
    }
    int ex, ey, tx, ty;
    block_scan_pair(local, local_runs, tmp, ex, ey, tx, ty);
    if (threadIdx.x == 0) {
        cnt[sb] = tx;
        if (RUNS && run_cnt) run_cnt[sb] = ty;
    }
}

// Column records of one chunk of columns, for the flat emission: offsets, the
// l interval and gap, (h, k), and the column's |g|^2 as a polynomial in l,
// q(l) = t + u l + G*33 l^2 with t = G*11 h^2 + G*22 k^2 + 2 G*12 hk and
// u = 2 G*13 h + 2 G*23 k in two-float arithmetic (about 1e-14 relative).
struct ChunkCols {
    int* off;   // [m + 1] exclusive reflection offsets within the chunk
    int* roff;  // [m + 1] exclusive run offsets
    int* a;     // first l
    int* c;     // first l of the inner gap (INT_MAX: none)
    int* gap;   // its length
    int* hk;    // (h << 16) | (k & 0xffff)
    float *th, *tl, *uh, *ul;
};

__device__ __forceinline__ ChunkCols chunk_cols(int* b, int m)
{
    ChunkCols cc;
    cc.off = b;
    cc.roff = b + (m + 1);
    int* r = b + 2 * (m + 1);
    cc.a = r;
    cc.c = r + m;
    cc.gap = r + 2 * m;
    cc.hk = r + 3 * m;
    cc.th = (float*)(r + 4 * m);
    cc.tl = (float*)(r + 5 * m);
    cc.uh = (float*)(r + 6 * m);
    cc.ul = (float*)(r + 7 * m);
    return cc;
}

__device__ __forceinline__ void put_col(const ChunkCols& cc, int i, const Geo& g, const ColSpan& sp, int h, int k)
{
    cc.a[i] = sp.a;
    cc.c[i] = sp.c <= sp.d ? sp.c : INT_MAX;
    cc.gap[i] = sp.c <= sp.d ? sp.d - sp.c + 1 : 0;
    cc.hk[i] = (h << 16) | (k & 0xffff);
    const F2 G11{g.gf[0], g.gl[0]}, G22{g.gf[1], g.gl[1]}, G12{2.f * g.gf[3], 2.f * g.gl[3]};
    const F2 G13{2.f * g.gf[4], 2.f * g.gl[4]}, G23{2.f * g.gf[5], 2.f * g.gl[5]};
    const F2 t = f2_add(f2_add(f2_mul_int(G11, (float)(h * h)), f2_mul_int(G22, (float)(k * k))),
                        f2_mul_int(G12, (float)(h * k)));
    const F2 u = f2_add(f2_mul_int(G13, (float)h), f2_mul_int(G23, (float)k));
    cc.th[i] = t.hi;
    cc.tl[i] = t.lo;
    cc.uh[i] = u.hi;
    cc.ul[i] = u.lo;
}

// Writes the chunk's reflections (and runs): thread t of nt takes positions t,
// t + nt, ...; each finds its column by bisection over the m offsets, so the
// writes of consecutive threads are consecutive.
template <bool RUNS>
__device__ __forceinline__ void emit_chunk(const F2 g33, const ChunkCols& cc, int m, int tot, int rtot, int t, int nt,
                                           int rb, int64_t base, int64_t cap, int done, int done_runs,
                                           double* __restrict__ q, uint32_t* __restrict__ key, int* __restrict__ runs)
{
    for (int p = t; p < tot; p += nt) {
        int lo = 0, hi = m - 1;  // last column with off <= p
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cc.off[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        const int hk = cc.hk[lo];
        int l = cc.a[lo] + (p - cc.off[lo]);
        if (l >= cc.c[lo]) l += cc.gap[lo];
        const int64_t pos = done + p;
        if (pos < cap) {
            const float fl = (float)l;
            const F2 v = f2_add(f2_add(F2{cc.th[lo], cc.tl[lo]}, f2_mul_int(g33, fl * fl)),
                                f2_mul_int(F2{cc.uh[lo], cc.ul[lo]}, fl));
            q[base + pos] = f2d_fast(v.hi) + f2d_fast(v.lo);
            key[base + pos] = hkl_pack(hk >> 16, (int)(short)(hk & 0xffff), l);
        }
    }
    if (RUNS) {
        for (int p = t; p < rtot; p += nt) {
            int lo = 0, hi = m - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (cc.roff[mid] <= p) lo = mid;
                else hi = mid - 1;
            }
            const int n = cc.off[lo + 1] - cc.off[lo];
            const int n1 = cc.gap[lo] > 0 ? cc.c[lo] - cc.a[lo] : n;
            const int j = p - cc.roff[lo], r1 = runs_of(n1, rb);
            const int first = j < r1 ? j * rb : n1 + (j - r1) * rb;
            const int len = j < r1 ? min(rb, n1 - j * rb) : min(rb, n - n1 - (j - r1) * rb);
            const int64_t rpos = done_runs + p;
            if (rpos < cap) runs[base + rpos] = ((done + cc.off[lo] + first) << 3) | len;
        }
    }
}

// The structure's entries of the structure-factor tile table from tile_off[s]:
// (s, first run) of each tile of 32 runs (rb > 0), or (s, first reflection)
// of each tile of tile_refl reflections.
__device__ __forceinline__ void write_tiles(int s, int rb, int tile_refl, int64_t units, const int* __restrict__ tile_off,
                                            int2* __restrict__ tile_tab, int t, int nt)
{
    const int per = rb > 0 ? kRunsPerTile : tile_refl;
    const int ntl = (int)((units + per - 1) / per), t0 = tile_off[s];
    for (int i = t; i < ntl; i += nt) tile_tab[t0 + i] = make_int2(s, i * per);
}

// Writes |g|^2 and the packed (h, k, l) of every reflection of each structure
// (and its runs, rb > 0) from refl_off[s], and its tile-table entries. The
// columns are taken 32 (one warp) or blockDim (the CTA) at a time: each thread
// finds its column's span, a scan places the columns, and the warp or CTA then
// writes the chunk's reflections and runs as one flat, coalesced range. The
// output order is the column order above, l ascending, whatever the launch shape.
// With one warp per structure the warps claim structures from ctr[0]; given the
// post-processing size-class lists (cls_list, cls_cnt), the structures above
// kPostCap6 reflections (the two largest classes) are left to whole CTAs,
// which claim them from ctr[1] once the warps are done. ctr: zero at launch.
// Dynamic shared memory: enum_smem_bytes(blockDim).
template <bool RUNS>
__global__ void __launch_bounds__(kEnumMaxThreads) k_emit(const Geo* __restrict__ geo, int n_struct, double r2min,
                                                          double r2max, float r2minf, float r2maxf, int rb,
                                                          int tile_refl, const int64_t* __restrict__ refl_off,
                                                          const int64_t* __restrict__ run_cnt,
                                                          const int* __restrict__ abort_flag, double* __restrict__ q,
                                                          uint32_t* __restrict__ key, int* __restrict__ runs,
                                                          const int* __restrict__ tile_off, int2* __restrict__ tile_tab,
                                                          int* __restrict__ ctr, const int* __restrict__ cls_list,
                                                          const int* __restrict__ cls_cnt)
{
    pdl_enter();
    extern __shared__ int esm[];
    __shared__ int tmp[66];
    __shared__ int s_big;
    if (*abort_flag) return;
    const int nt = blockDim.x, t = threadIdx.x;
    const bool per_warp = enum_per_warp(nt);
    const int w = t >> 5, lane = t & 31;
    const int64_t big_min = cls_list ? kPostCap6 : INT64_MAX;
    int nbig = 0;
    if (per_warp) {
        const ChunkCols cc = chunk_cols(esm + enum_cta_ints(nt) + w * kWarpRecInts, 32);
        for (;;) {
            int s = 0;
            if (lane == 0) s = atomicAdd(ctr, 1);
            s = __shfl_sync(0xffffffffu, s, 0);
            if (s >= n_struct) break;
            const int64_t base = refl_off[s], cap = refl_off[s + 1] - base;
            if (tile_tab) write_tiles(s, rb, tile_refl, rb > 0 ? run_cnt[s] : cap, tile_off, tile_tab, lane, 32);
            if (cap <= 0 || cap > big_min) continue;
            const Geo g = geo[s];
            const F2 g33{g.gf[2], g.gl[2]};
            const int ncol = n_columns(g);
            int done = 0, done_runs = 0;
            for (int c0 = 0; c0 < ncol; c0 += 32) {
                const int c = c0 + lane;
                int m = 0, mr = 0;
                if (c < ncol) {
                    int h, k;
                    const ColSpan sp =
                        column_counts(g, geo[s].gs, c, r2min, r2max, r2minf, r2maxf, rb, RUNS, h, k, m, mr);
                    put_col(cc, lane, g, sp, h, k);
                }
                const int im = warp_incl_scan(m), imr = RUNS ? warp_incl_scan(mr) : 0;
                cc.off[lane] = im - m;
                if (RUNS) cc.roff[lane] = imr - mr;
                const int tot = __shfl_sync(0xffffffffu, im, 31);
                const int rtot = RUNS ? __shfl_sync(0xffffffffu, imr, 31) : 0;
                if (lane == 0) {
                    cc.off[32] = tot;
                    cc.roff[32] = rtot;
                }
                __syncwarp();
                emit_chunk<RUNS>(g33, cc, 32, tot, rtot, lane, 32, rb, base, cap, done, done_runs, q, key, runs);
                done += tot;
                done_runs += rtot;
                __syncwarp();  // the records are read before the next chunk rewrites them
            }
        }
        if (!cls_list) return;
        nbig = cls_cnt[kPostFlatClass - 1] + cls_cnt[kPostFlatClass];
        if (nbig == 0) return;
    }
    const ChunkCols cc = chunk_cols(esm, nt);
    for (int it = 0;; it++) {  // the structures taken by the whole CTA
        int sb;
        if (per_warp) {
            __syncthreads();  // s_big and the chunk records are free
            if (t == 0) s_big = atomicAdd(ctr + 1, 1);
            __syncthreads();
            const int j = s_big;
            if (j >= nbig) break;
            const int n5 = cls_cnt[kPostFlatClass];  // the largest class first
            sb = j < n5 ? cls_list[(int64_t)kPostFlatClass * n_struct + j]
                        : cls_list[(int64_t)(kPostFlatClass - 1) * n_struct + (j - n5)];
        } else {
            if (it > 0) break;
            sb = blockIdx.x;  // one CTA per structure
            if (sb >= n_struct) break;
        }
        const int64_t base = refl_off[sb], capb = refl_off[sb + 1] - base;
        if (!per_warp && tile_tab) write_tiles(sb, rb, tile_refl, rb > 0 ? run_cnt[sb] : capb, tile_off, tile_tab, t, nt);
        if (capb <= 0) continue;
        const Geo g = geo[sb];
        const F2 g33{g.gf[2], g.gl[2]};
        const int ncol = n_columns(g);
        int done = 0, done_runs = 0;
        for (int c0 = 0; c0 < ncol; c0 += nt) {
            const int c = c0 + t;
            int m = 0, mr = 0;
            if (c < ncol) {
                int h, k;
                const ColSpan sp =
                    column_counts(g, geo[sb].gs, c, r2min, r2max, r2minf, r2maxf, rb, RUNS, h, k, m, mr);
                put_col(cc, t, g, sp, h, k);
            }
            int ex, ey, tx, ty;
            block_scan_pair(m, mr, tmp, ex, ey, tx, ty);
            cc.off[t] = ex;
            cc.roff[t] = ey;
            if (t == 0) {
                cc.off[nt] = tx;
                cc.roff[nt] = ty;
            }
            __syncthreads();
            emit_chunk<RUNS>(g33, cc, nt, tx, ty, t, nt, rb, base, capb, done, done_runs, q, key, runs);
            done += tx;
            done_runs += ty;
            __syncthreads();  // the chunk's records are read; the next chunk rewrites them
        }
    }
}

// Single block. Every pass walks the batch in chunks of kScanItems * blockDim
// structures (or positions in the largest-first order): coalesced loads into
// registers, a transpose through shared memory when a pass needs a prefix,
// and warp-aggregated shared-memory atomics where it needs ranks.
//  1. reflection offsets (64-bit exclusive scan of the counts), the capacity
//     check and the per-structure status;
//  2. in the largest-first order (k_order), each structure's first tile and
//     the post-processing size-class lists (post_class; within a class the
//     order follows the chunks).
// The tile table itself is written by k_emit, one CTA per structure.
constexpr int kOrderBins = 4096;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;

__device__ __forceinline__ int order_bin(const int64_t* __restrict__ atom_off, int s)
{
    const long long na = atom_off[s + 1] - atom_off[s];
    return kOrderBins - 1 - (int)min(max(na, 0LL), (long long)(kOrderBins - 1));
}

// Rank of this lane among the lanes of its warp with the same key, and the
// base the group's leader obtained with one shared-memory atomicAdd on ctr[key].
__device__ __forceinline__ int warp_aggregated_slot(int* ctr, int key, bool active)
{
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (!active) return 0;
    const unsigned peers = __match_any_sync(act, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&ctr[key], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}

__global__ void __launch_bounds__(kScanThreads) k_scan_refl(const int64_t* __restrict__ cnt,
                                                            const int64_t* __restrict__ run_cnt,
                                                            const Geo* __restrict__ geo, int n, int tile_refl,
                                                            int64_t cap_refl, int64_t* __restrict__ refl_off,
                                                            int* __restrict__ tile_off, const int* __restrict__ order,
                                                            int* __restrict__ cls_list, int* __restrict__ abort_flag,
                                                            int64_t* __restrict__ totals, int32_t* __restrict__ status,
                                                            unsigned long long* __restrict__ work)
{
    pdl_enter();
    __shared__ long long ws[33];
    __shared__ __align__(16) long long buf[kScanItems * kScanThreads];
    __shared__ int ccnt[kPostClasses];
    const int nt = blockDim.x, tid = threadIdx.x, CH = kScanItems * nt;
    long long tot;
    // 1. reflection offsets in structure order, and the status of each structure
    long long carry = 0, bad = 0;
    for (int base = 0; base < n; base += CH) {
        long long v[kScanItems];
        int st[kScanItems];
#pragma unroll
        for (int u = 0; u < kScanItems; u++) {
            const int i = base + u * nt + tid;
            v[u] = i < n ? cnt[i] : 0;
            st[u] = i < n ? geo[i].status : XRD_OK;
        }
        chunk_scan<kScanItems>(v, buf, ws, &tot);
#pragma unroll
        for (int u = 0; u < kScanItems; u++) {
            const int i = base + u * nt + tid;
            if (i < n) {
                refl_off[i] = carry + v[u];
                status[i] = st[u];
            }
            bad += st[u] != XRD_OK;
        }
        carry += tot;
    }
    const long long total = carry;
    const bool over = total > cap_refl;
    block_prefix_ll(bad, ws, &tot);
    const long long nbad = over ? n : tot;
    if (over)
        for (int i = tid; i < n; i += nt) status[i] = XRD_ECAPACITY;
    if (tid < kPostClasses) ccnt[tid] = 0;
    __syncthreads();
    // 2. tiles and size classes in the largest-first order
    long long tcarry = 0;
    for (int base = 0; base < n; base += CH) {
        long long v[kScanItems];
        int sv[kScanItems];
#pragma unroll
        for (int u = 0; u < kScanItems; u++) {
            const int p = base + u * nt + tid;
            sv[u] = p < n ? order[p] : -1;
        }
        long long c[kScanItems];
#pragma unroll
        for (int u = 0; u < kScanItems; u++) {
            c[u] = sv[u] >= 0 ? cnt[sv[u]] : 0;
            // tiles of 32 runs, or of tile_refl reflections
            v[u] = sv[u] < 0 ? 0 : (tile_refl > 0 ? (c[u] + tile_refl - 1) / tile_refl
                                                  : (run_cnt[sv[u]] + kRunsPerTile - 1) / kRunsPerTile);
        }
        chunk_scan<kScanItems>(v, buf, ws, &tot);
#pragma unroll
        for (int u = 0; u < kScanItems; u++) {
            const int p = base + u * nt + tid;
            if (p < n) tile_off[sv[u]] = (int)(tcarry + v[u]);  // first tile of the structure
            if (!over && cls_list) {
                const int k = post_class(c[u]);
                const int slot = warp_aggregated_slot(ccnt, k, p < n);
                if (p < n) cls_list[(int64_t)k * n + slot] = sv[u];
            }
        }
        tcarry += tot;
        __syncthreads();  // this chunk's class slots are taken before the next chunk's
    }
    if (tid == 0) {
        if (work) {  // for xrd_work_counts: the tiles and the tile mode of this call
            work[0] = (unsigned long long)tcarry;
            work[1] = tile_refl > 0 ? 0ull : 1ull;
        }
        refl_off[n] = total;
        tile_off[n] = over ? 0 : (int)tcarry;
        for (int k = 0; k < kPostClasses; k++) abort_flag[kFlagClsCnt + k] = over ? 0 : ccnt[k];
        totals[0] = total;
        totals[1] = 0;
        totals[2] = 0;
        totals[3] = nbad;
        *abort_flag = over;
    }
}

// Multi-block form of k_scan_refl for batches of more than two chunks (one
// chunk of kScanItems * kScanThreads structures per CTA): k_scan_refl_parts
// writes each chunk's sums (reflections, invalid structures, tiles in the
// largest-first order, structures per size class); k_scan_refl_final offsets
// every chunk by the sums of the chunks before it and repeats the single-block
// passes on its own chunk. Class-list slots follow the chunk order.
constexpr int kScanPartWords = 3 + kPostClasses;  // refl, bad, tiles, class counts

__device__ __forceinline__ long long tiles_of(const int64_t* __restrict__ run_cnt, int s, long long c, int tile_refl)
{
    return tile_refl > 0 ? (c + tile_refl - 1) / tile_refl : (run_cnt[s] + kRunsPerTile - 1) / kRunsPerTile;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_refl_parts(const int64_t* __restrict__ cnt,
                                                                  const int64_t* __restrict__ run_cnt,
                                                                  const Geo* __restrict__ geo, int n, int tile_refl,
                                                                  const int* __restrict__ order,
                                                                  long long* __restrict__ parts)
{
    pdl_enter();
    __shared__ long long ws[33];
    __shared__ int cc[kPostClasses];
    const int nt = blockDim.x, tid = threadIdx.x, base = blockIdx.x * kScanItems * nt;
    if (tid < kPostClasses) cc[tid] = 0;
    __syncthreads();
    long long refl = 0, bad = 0, tiles = 0;
#pragma unroll
    for (int u = 0; u < kScanItems; u++) {
        const int i = base + u * nt + tid;
        if (i < n) {
            refl += cnt[i];
            bad += geo[i].status != XRD_OK;
            const int sv = order[i];  // position i of the largest-first order
            const long long c = cnt[sv];
            tiles += tiles_of(run_cnt, sv, c, tile_refl);
            atomicAdd(&cc[post_class(c)], 1);
        }
    }
    long long t;
    block_prefix_ll(refl, ws, &t);
    refl = t;
    block_prefix_ll(bad, ws, &t);
    bad = t;
    block_prefix_ll(tiles, ws, &t);
    tiles = t;
    if (tid == 0) {
        long long* o = parts + (int64_t)blockIdx.x * kScanPartWords;
        o[0] = refl;
        o[1] = bad;
        o[2] = tiles;
        for (int k = 0; k < kPostClasses; k++) o[3 + k] = cc[k];
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_refl_final(const int64_t* __restrict__ cnt,
                                                                  const int64_t* __restrict__ run_cnt,
                                                                  const Geo* __restrict__ geo, int n, int tile_refl,
                                                                  int64_t cap_refl, int64_t* __restrict__ refl_off,
                                                                  int* __restrict__ tile_off, const int* __restrict__ order,
                                                                  int* __restrict__ cls_list, int* __restrict__ abort_flag,
                                                                  int64_t* __restrict__ totals, int32_t* __restrict__ status,
                                                                  unsigned long long* __restrict__ work,
                                                                  const long long* __restrict__ parts)
{
    pdl_enter();
    __shared__ long long ws[33];
    __shared__ __align__(16) long long buf[kScanItems * kScanThreads];
    __shared__ long long pre[kScanPartWords], all[kScanPartWords];
    __shared__ int ccnt[kPostClasses];
    const int nt = blockDim.x, tid = threadIdx.x, b = blockIdx.x, base = b * kScanItems * nt;
    const int nch = gridDim.x;
    if (tid < kScanPartWords) {  // sums of the chunks before this one, and of all chunks
        long long p = 0, a = 0;
        for (int c = 0; c < nch; c++) {
            const long long v = parts[(int64_t)c * kScanPartWords + tid];
            p += c < b ? v : 0;
            a += v;
        }
        pre[tid] = p;
        all[tid] = a;
    }
    if (tid < kPostClasses) ccnt[tid] = 0;
    __syncthreads();
    const long long total = all[0];
    const bool over = total > cap_refl;
    long long v[kScanItems], tot;
    int st[kScanItems];
    // 1. reflection offsets and status
#pragma unroll
    for (int u = 0; u < kScanItems; u++) {
        const int i = base + u * nt + tid;
        v[u] = i < n ? cnt[i] : 0;
        st[u] = i < n ? geo[i].status : XRD_OK;
    }
    chunk_scan<kScanItems>(v, buf, ws, &tot);
#pragma unroll
    for (int u = 0; u < kScanItems; u++) {
        const int i = base + u * nt + tid;
        if (i < n) {
            refl_off[i] = pre[0] + v[u];
            status[i] = over ? XRD_ECAPACITY : st[u];
        }
    }
    // 2. first tile of each structure and the size-class lists, in the largest-first order
    int sv[kScanItems];
    long long c[kScanItems];
#pragma unroll
    for (int u = 0; u < kScanItems; u++) {
        const int p = base + u * nt + tid;
        sv[u] = p < n ? order[p] : -1;
        c[u] = sv[u] >= 0 ? cnt[sv[u]] : 0;
        v[u] = sv[u] < 0 ? 0 : tiles_of(run_cnt, sv[u], c[u], tile_refl);
    }
    chunk_scan<kScanItems>(v, buf, ws, &tot);
#pragma unroll
    for (int u = 0; u < kScanItems; u++) {
        const int p = base + u * nt + tid;
        if (p < n) tile_off[sv[u]] = (int)(pre[2] + v[u]);
        if (!over && cls_list) {
            const int k = post_class(c[u]);
            const int slot = warp_aggregated_slot(ccnt, k, p < n);
            if (p < n) cls_list[(int64_t)k * n + (int)pre[3 + k] + slot] = sv[u];
        }
    }
    if (b == 0 && tid == 0) {
        if (work) {
            work[0] = (unsigned long long)all[2];
            work[1] = tile_refl > 0 ? 0ull : 1ull;
        }
        refl_off[n] = total;
        tile_off[n] = over ? 0 : (int)all[2];
        for (int k = 0; k < kPostClasses; k++) abort_flag[kFlagClsCnt + k] = over ? 0 : (int)all[3 + k];
        totals[0] = total;
        totals[1] = 0;
        totals[2] = 0;
        totals[3] = over ? n : all[1];
        *abort_flag = over;
    }
}

// Largest-first order of the structures: a counting sort on the atom count
// (which sets the cost of a structure-factor tile), in descending order; one
// block, warp-aggregated shared-memory atomics, so structures of one bin keep
// the order of their warp. It depends on the input only and runs beside the
// enumeration.
__global__ void __launch_bounds__(kScanThreads) k_order(const int64_t* __restrict__ atom_off, int n,
                                                        int* __restrict__ order)
{
    pdl_enter();
    __shared__ int bins[kOrderBins];
    __shared__ int tmp[66];
    const int nt = blockDim.x, tid = threadIdx.x, CH = kScanItems * nt;
    for (int b = tid; b < kOrderBins; b += nt) bins[b] = 0;
    __syncthreads();
    for (int base = 0; base < n; base += CH) {
        int b[kScanItems];
#pragma unroll
        for (int u = 0; u < kScanItems; u++) {
            const int i = base + u * nt + tid;
            b[u] = i < n ? order_bin(atom_off, i) : 0;
        }
#pragma unroll
        for (int u = 0; u < kScanItems; u++) warp_aggregated_slot(bins, b[u], base + u * nt + tid < n);
    }
    __syncthreads();
    block_excl_scan(bins, kOrderBins, tmp);
    for (int base = 0; base < n; base += CH) {
        int b[kScanItems];
#pragma unroll
        for (int u = 0; u < kScanItems; u++) {
            const int i = base + u * nt + tid;
            b[u] = i < n ? order_bin(atom_off, i) : 0;
        }
#pragma unroll
        for (int u = 0; u < kScanItems; u++) {
            const int i = base + u * nt + tid;
            const int slot = warp_aggregated_slot(bins, b[u], i < n);
            if (i < n) order[slot] = i;
        }
    }
}

// Multi-block form of the same order (more than two chunks of kScanItems *
// kScanThreads structures). k_order_parts histograms each chunk into
// oparts[chunk][bin]; k_order_final starts each bin of a chunk after all
// structures of the earlier bins and those of the same bin in earlier chunks,
// then scatters the chunk as k_order does.
__global__ void __launch_bounds__(kScanThreads) k_order_parts(const int64_t* __restrict__ atom_off, int n,
                                                              int* __restrict__ oparts)
{
    pdl_enter();
    __shared__ int bins[kOrderBins];
    const int nt = blockDim.x, tid = threadIdx.x, base = blockIdx.x * kScanItems * nt;
    for (int b = tid; b < kOrderBins; b += nt) bins[b] = 0;
    __syncthreads();
    int b[kScanItems];
#pragma unroll
    for (int u = 0; u < kScanItems; u++) {
        const int i = base + u * nt + tid;
        b[u] = i < n ? order_bin(atom_off, i) : 0;
    }
#pragma unroll
    for (int u = 0; u < kScanItems; u++) warp_aggregated_slot(bins, b[u], base + u * nt + tid < n);
    __syncthreads();
    for (int j = tid; j < kOrderBins; j += nt) oparts[(size_t)blockIdx.x * kOrderBins + j] = bins[j];
}

__global__ void __launch_bounds__(kScanThreads) k_order_final(const int64_t* __restrict__ atom_off, int n,
                                                              const int* __restrict__ oparts, int* __restrict__ order)
{
    pdl_enter();
    __shared__ int bins[kOrderBins], before[kOrderBins];
    __shared__ int tmp[66];
    const int nt = blockDim.x, tid = threadIdx.x, ch = blockIdx.x, nch = gridDim.x, base = ch * kScanItems * nt;
    for (int j = tid; j < kOrderBins; j += nt) {
        int tot = 0, bef = 0;
        for (int c = 0; c < nch; c++) {
            const int v = oparts[(size_t)c * kOrderBins + j];
            tot += v;
            bef += c < ch ? v : 0;
        }
        bins[j] = tot;
        before[j] = bef;
    }
    __syncthreads();
    block_excl_scan(bins, kOrderBins, tmp);
    for (int j = tid; j < kOrderBins; j += nt) bins[j] += before[j];
    __syncthreads();
    int b[kScanItems];
#pragma unroll
    for (int u = 0; u < kScanItems; u++) {
        const int i = base + u * nt + tid;
        b[u] = i < n ? order_bin(atom_off, i) : 0;
    }
#pragma unroll
    for (int u = 0; u < kScanItems; u++) {
        const int i = base + u * nt + tid;
        const int slot = warp_aggregated_slot(bins, b[u], i < n);
        if (i < n) order[slot] = i;
    }
}

template <typename... P, typename... A>
static void launch_k(bool pdl, void (*k)(P...), dim3 grid, dim3 block, cudaStream_t st, A... args)
{
    if (pdl) launch_pdl(k, grid, block, 0, st, args...);
    else k<<<grid, block, 0, st>>>(static_cast<P>(args)...);
}

static void prep_launch(bool pdl, const double* lattice, int n, double rmax, Geo* geo, unsigned* imax,
                        int32_t* flags, cudaStream_t st)
{
    if (n <= kPrepWideMax)  // 4 structures per CTA
        launch_k(pdl, k_prep<8>, (n + 3) / 4, 32, st, lattice, n, rmax, geo, imax, flags);
    else launch_k(pdl, k_prep<1>, (n + 127) / 128, 128, st, lattice, n, rmax, geo, imax, flags);
}

// Structure-factor work of the last call (for xrd_work_counts): terms = sum of
// reflections x atoms; phase seeds = the same with strided tiles, runs x atoms
// with runs; out[0..2] = terms, seeds, tiles (out zeroed by the caller).
__global__ void __launch_bounds__(256) k_work(const int64_t* __restrict__ cnt, const int64_t* __restrict__ run_cnt,
                                              const int64_t* __restrict__ atom_off, int n,
                                              const unsigned long long* __restrict__ work,
                                              unsigned long long* __restrict__ out)
{
    __shared__ unsigned long long red[2][8];
    const bool runs = work[1] != 0;
    unsigned long long t = 0, sd = 0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const unsigned long long na = (unsigned long long)(atom_off[s + 1] - atom_off[s]);
        t += (unsigned long long)cnt[s] * na;
        sd += (unsigned long long)(runs ? run_cnt[s] : cnt[s]) * na;
    }
    for (int o = 16; o > 0; o >>= 1) {
        t += __shfl_xor_sync(0xffffffffu, t, o);
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = t;
        red[1][w] = sd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); i++) {
            t += red[0][i];
            sd += red[1][i];
        }
        atomicAdd(&out[0], t);
        atomicAdd(&out[1], sd);
        if (blockIdx.x == 0) out[2] = work[0];
    }
}

void launch_work(const GeomArgs& a, unsigned long long* out, cudaStream_t st)
{
    if (a.n_struct > 0)
        k_work<<<min((a.n_struct + 255) / 256, 1024), 256, 0, st>>>(a.refl_cnt, a.run_cnt, a.atom_off, a.n_struct,
                                                                   a.work, out);
}

void launch_prep(const GeomArgs& a, cudaStream_t st, bool pdl)
{
    if (a.n_struct > 0) prep_launch(pdl, a.lattice, a.n_struct, a.rmax, a.geo, a.imax, a.out_flags, st);
}

void launch_coef(const GeomArgs& a, cudaStream_t st, bool pdl)
{
    launch_k(pdl, k_coef, 1, 256, st, a.coef, a.zmax, a.coef32, a.cdd);
}

void launch_atoms(const GeomArgs& a, cudaStream_t st, bool pdl)
{
    if (a.n_struct > 0)
        launch_k(pdl, k_atoms, a.n_struct, 128, st, a.atom_off, a.n_atoms, a.frac, a.Z, a.occ, a.B, a.zmax, a.geo,
                 a.atoms_set_geo, a.atom_bad, a.atom32, a.atom64, a.runs_mode ? a.astep : (float2*)nullptr, a.atomr,
                 a.sctab);
}

void launch_order(const GeomArgs& a, cudaStream_t st, bool pdl)
{
    if (a.n_struct <= 0) return;
    const int nch = (a.n_struct + kScanItems * kScanThreads - 1) / (kScanItems * kScanThreads);
    if (nch <= 2 || !a.oparts) {
        launch_k(pdl, k_order, 1, kScanThreads, st, a.atom_off, a.n_struct, a.order);
        return;
    }
    launch_k(pdl, k_order_parts, nch, kScanThreads, st, a.atom_off, a.n_struct, a.oparts);
    launch_k(true, k_order_final, nch, kScanThreads, st, a.atom_off, a.n_struct, (const int*)a.oparts, a.order);
}

size_t order_parts_bytes(int64_t n)
{
    const int64_t nch = (n + kScanItems * kScanThreads - 1) / (kScanItems * kScanThreads);
    return nch > 2 ? (size_t)4 * kOrderBins * nch : 0;
}

void launch_count_only(const GeomArgs& a, cudaStream_t st)
{
    const int n = a.n_struct;
    if (n <= 0) return;
    prep_launch(false, a.lattice, n, a.rmax, a.geo, (unsigned*)nullptr, (int32_t*)nullptr, st);
    launch_pdl(k_count<false>, (n + 7) / 8, 256, 0, st, a.geo, n, a.r2min,
               a.r2max, (float)a.r2min, (float)a.r2max, 0, a.refl_cnt, (int64_t*)nullptr, a.enum_ctr);
}

static int enum_grid(const GeomArgs& a)
{
    const int per = enum_per_warp(a.enum_threads) ? a.enum_threads / 32 : 1;  // structures per CTA
    return (a.n_struct + per - 1) / per;
}

void launch_count(const GeomArgs& a, cudaStream_t st, bool pdl)
{
    if (a.n_struct > 0)
        launch_k(pdl, a.runs_mode ? k_count<true> : k_count<false>, enum_grid(a), a.enum_threads, st, a.geo,
                 a.n_struct, a.r2min, a.r2max,
                 (float)a.r2min, (float)a.r2max, a.runs_mode ? a.rb : 0, a.refl_cnt, a.run_cnt, a.enum_ctr);
}

int scan_chunks(int n) { return (n + kScanItems * kScanThreads - 1) / (kScanItems * kScanThreads); }

void launch_scan_refl(const GeomArgs& a, cudaStream_t st, bool pdl)
{
    const int nch = scan_chunks(a.n_struct);
    const int tile_refl = a.runs_mode ? 0 : 32 * a.rb;
    if (nch <= 2 || !a.parts) {  // one block walks the chunks
        launch_k(pdl, k_scan_refl, 1, kScanThreads, st, a.refl_cnt, a.run_cnt, a.geo, a.n_struct, tile_refl,
                 a.cap_refl, a.refl_off, a.tile_off, (const int*)a.order, a.cls_list, a.abort_flag, a.totals,
                 a.status, a.work);
        return;
    }
    launch_k(pdl, k_scan_refl_parts, nch, kScanThreads, st, a.refl_cnt, a.run_cnt, a.geo, a.n_struct, tile_refl,
             (const int*)a.order, a.parts);
    launch_k(true, k_scan_refl_final, nch, kScanThreads, st, a.refl_cnt, a.run_cnt, a.geo, a.n_struct, tile_refl,
             a.cap_refl, a.refl_off, a.tile_off, (const int*)a.order, a.cls_list, a.abort_flag, a.totals, a.status,
             a.work, (const long long*)a.parts);
}

void launch_emit(const GeomArgs& a, cudaStream_t st, bool pdl)
{
    if (a.n_struct <= 0) return;
    auto k = a.runs_mode ? k_emit<true> : k_emit<false>;
    const size_t smem = enum_smem_bytes(a.enum_threads);
    if (pdl)
        launch_pdl(k, enum_grid(a), a.enum_threads, smem, st, a.geo, a.n_struct, a.r2min, a.r2max, (float)a.r2min,
                   (float)a.r2max, a.runs_mode ? a.rb : 0, 32 * a.rb, (const int64_t*)a.refl_off,
                   (const int64_t*)a.run_cnt, (const int*)a.abort_flag, a.q, a.key, a.runs, (const int*)a.tile_off,
                   a.tile_tab, a.enum_ctr + 1, (const int*)a.cls_list, (const int*)(a.abort_flag + kFlagClsCnt));
    else
        k<<<enum_grid(a), a.enum_threads, smem, st>>>(a.geo, a.n_struct, a.r2min, a.r2max, (float)a.r2min,
                                                       (float)a.r2max, a.runs_mode ? a.rb : 0, 32 * a.rb,
                                                       a.refl_off, a.run_cnt, a.abort_flag, a.q, a.key, a.runs,
                                                       a.tile_off, a.tile_tab, a.enum_ctr + 1, a.cls_list,
                                                       a.abort_flag + kFlagClsCnt);
}

}  // namespace xrd
