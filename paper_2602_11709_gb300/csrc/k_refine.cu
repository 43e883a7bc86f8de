// Accurate re-evaluation of the reflections whose FP32 intensity is not
// accurate enough (FP32 pattern variants, between steps S3 and S4).
//
// The FP32 structure-factor pass rounds every term: sin/cos (MUFU, about 1e-7
// absolute), the Debye-Waller and f(s) exponentials (MUFU ex2, about 5e-8
// relative) and the blocked sum. Each term's error scales with
// a_j = occ_j exp(-B_j s^2) max(|f_j|, Z_j), and the errors of different atoms
// are independent, so |F| errs by about eps sqrt(sum_j a_j^2) (eps: the
// per-term error) whatever |F| is. A weak reflection (|F| much below that
// root-sum-square, the destructive interference of many atoms) then has a
// large relative error in I = |F|^2 LP. The agreement the engine promises is
// relative per kept peak (Sec. 3 compares peak intensities), so such
// reflections are evaluated again here, term by term, in double-float
// arithmetic (two FP32 numbers, about 48 bits) from exact 64-bit fixed-point
// phases, with per-term errors near 1e-11.
//
// Which reflections: with dF = eps_k sqrt(sum a_j^2) (eps_k = K eps, a
// K-sigma bound) the intensity's error bound is E = LP (2 |F| dF + dF^2). A
// reflection is re-evaluated when E > tau max(I, c M), M the structure's
// largest reflection intensity and c the cutoff fraction (1e-3 when the cutoff
// is off). Every other reflection then errs by at most tau of its own
// intensity, or by at most tau c M: a peak kept by the cutoff (above c times
// the largest peak, itself at least 2 M) errs by at most tau times its
// intensity per member of that kind.
#include "xrd_dd.cuh"
#include "xrd_launch.h"

namespace xrd {

static __device__ float4 g_sc_tab[256];  // cos and sin of 2 pi k / 256 as two floats each
static __device__ float2 g_ex_tab[64];   // 2^(-j / 64) as two floats

__global__ void k_refine_tab_init()
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 256) {
        double sn, cs;
        sincospi(k / 128.0, &sn, &cs);
        const DD c = dd_from_double(cs), s = dd_from_double(sn);
        g_sc_tab[k] = make_float4(c.hi, c.lo, s.hi, s.lo);
    }
    if (k < 64) {
        const DD e = dd_from_double(exp2(-k / 64.0));
        g_ex_tab[k] = make_float2(e.hi, e.lo);
    }
}

RefineTables init_refine_tables(cudaStream_t st)
{
    RefineTables t{};
    k_refine_tab_init<<<1, 256, 0, st>>>();
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sc_tab) != cudaSuccess) return RefineTables{};
    t.sc = (const float4*)p;
    if (cudaGetSymbolAddress(&p, g_ex_tab) != cudaSuccess) return RefineTables{};
    t.ex = (const float2*)p;
    return t;
}

// f(s) = Z - 41.78214 s^2 sum_i a_i exp(-b_i s^2) in double-float
__device__ __forceinline__ DD f_dd(const float4* __restrict__ cdd, int z, DD s2, const float2* __restrict__ ex)
{
    DD sum{0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float4 c = cdd[4 * z + i];
        const DD e = dd_exp_neg(dd_mul(DD{c.z, c.w}, s2), ex);
        sum = dd_add(sum, dd_mul(DD{c.x, c.y}, e));
    }
    constexpr float Fh = 41.78213882446289f, Fl = 1.1755371360777644e-06f;  // 41.78214
    const DD t = dd_mul(dd_mul(sum, s2), DD{Fh, Fl});
    return dd_add(DD{(float)z, 0.f}, dd_neg(t));
}

constexpr int kRefThreads = 256;  // also the reflections per work chunk
constexpr int kRefWarps = kRefThreads / 32;

// One warp re-evaluates reflection r of structure s: lanes take the
// structure's (element-sorted) atoms 32 at a time; in each batch of 32 the
// first lane of every run of one element evaluates f(s) and hands it to the
// run's other lanes; then a two-float reduction across the warp, and lane 0
// writes I = |F|^2 LP (LP in FP64).
__device__ void refine_one(const RefineArgs& a, int64_t r, int s, const float4* ssc, const float2* sex)
{
    const int lane = threadIdx.x & 31;
    const double q = a.q[r];
    const uint32_t key = a.key[r];
    const long long h = hkl_h(key), k = hkl_k(key), l = hkl_l(key);
    float qh, ql;
    split_pos(q, qh, ql);                                // |g|^2 as two floats, no FP64 arithmetic
    const DD qd = dd_fast2sum(qh, ql);
    const DD s2 = dd_mul_f(qd, 0.25f);  // exact scaling
    const int64_t j0 = a.atom_off[s], j1 = a.atom_off[s + 1];
    DD Fr{0.f, 0.f}, Fi{0.f, 0.f};
    for (int64_t jb = j0; jb < j1; jb += 32) {
        const int64_t j = jb + lane;
        const bool live = j < j1;
        AtomR at{};
        if (live) at = a.atomr[j];
        const int z = live ? at.z : -1;
        const int zprev = __shfl_up_sync(0xffffffffu, z, 1);
        const bool head = live && (lane == 0 || zprev != z);
        const unsigned heads = __ballot_sync(0xffffffffu, head);
        DD f{0.f, 0.f};
        if (head) f = f_dd(a.cdd, z, s2, sex);
        const int src = 31 - __clz(heads & ((2u << lane) - 1u));  // the last run head at or below this lane
        f.hi = __shfl_sync(0xffffffffu, f.hi, src);
        f.lo = __shfl_sync(0xffffffffu, f.lo, src);
        if (live) {
            const unsigned long long P = (unsigned long long)h * at.X + (unsigned long long)k * at.Y +
                                         (unsigned long long)l * at.Z;
            DD cs, sn;
            dd_sincos_turn(P, ssc, cs, sn);
            const DD dw = dd_exp_neg(dd_mul(DD{at.bh, at.bl}, s2), sex);
            const DD w = dd_mul(dd_mul(DD{at.oh, at.ol}, f), dw);
            Fr = dd_add(Fr, dd_mul(w, cs));
            Fi = dd_add(Fi, dd_mul(w, sn));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DD tr{__shfl_xor_sync(0xffffffffu, Fr.hi, o), __shfl_xor_sync(0xffffffffu, Fr.lo, o)};
        const DD ti{__shfl_xor_sync(0xffffffffu, Fi.hi, o), __shfl_xor_sync(0xffffffffu, Fi.lo, o)};
        Fr = dd_add(Fr, tr);
        Fi = dd_add(Fi, ti);
    }
    if (lane == 0) {
        // |F|^2 in double-float; LP in FP32 from sin^2 theta = X as two floats, with
        // cos^2 theta = (1 - Xh) - Xl (1 - Xh exact for Xh >= 1/2): a few ulp whatever 2-theta
        const DD F2 = dd_add(dd_mul(Fr, Fr), dd_mul(Fi, Fi));
        const float Xh = qd.hi * a.l2h;
        const float Xl = fmaf(qd.hi, a.l2h, -Xh) + fmaf(qd.hi, a.l2l, qd.lo * a.l2h);
        const float X = Xh + Xl;
        const float u = fmaxf((1.f - Xh) - Xl, (float)kCos90Sq);
        const float c2 = fmaf(-2.f, X, 1.f);
        const float lp = fmaf(c2, c2, 1.f) / (X * sqrtf(u));
        a.If[r] = (F2.hi + F2.lo) * lp;
    }
}


// Selection: one streaming pass over the reflections (error bound and
// intensity, 8 bytes each). Every candidate has E > tau I (the criterion is
// E > tau max(I, c M)); for those few the structure-factor kernel has noted the
// structure, whose floor c M decides. Candidates are appended with one atomic
// per warp.
__device__ __forceinline__ bool refine_take(const RefineArgs& a, int64_t r, float E, float I, int& s)
{
    if (!(E > 0.f && E > a.tau * I)) return false;
    s = a.Es[r];
    const float floorI = a.cref * __uint_as_float(a.imax[s]);
    const bool bad = a.atom_bad && a.atom_bad[s];
    return !bad && E > a.tau * fmaxf(I, floorI);
}

// A CTA collects its candidates in shared memory and appends them to the list
// with one atomic per flush: candidates are rare (a fraction of a percent), and
// one atomic per warp on the list's single counter had serialised.
constexpr int kSelCap = 2048;  // shared-memory candidates per CTA; flushed above kSelCap - 4 kRefThreads

__global__ void __launch_bounds__(kRefThreads) k_refine_select(const RefineArgs a)
{
    pdl_enter();
    __shared__ int64_t sr[kSelCap];
    __shared__ int ss[kSelCap];
    __shared__ int sn;
    __shared__ unsigned long long sbase;
    if (*a.abort_flag) return;
    const int64_t total = a.refl_off[a.n_struct];
    if (threadIdx.x == 0) sn = 0;
    __syncthreads();
    auto flush = [&]() {
        const int m = sn;
        if (threadIdx.x == 0 && m > 0) sbase = atomicAdd(a.nref, (unsigned long long)m);
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += kRefThreads) {
            a.cand_r[sbase + i] = sr[i];
            a.cand_s[sbase + i] = ss[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) sn = 0;
        __syncthreads();
    };
    // the CTA takes 4 kRefThreads consecutive reflections at a time, four per thread in one 16-byte
    // load of each array (both 256-byte aligned)
    constexpr int kChunk = 4 * kRefThreads;
    for (int64_t c0 = (int64_t)blockIdx.x * kChunk; c0 < total; c0 += (int64_t)gridDim.x * kChunk) {
        const int64_t r4 = c0 + 4 * threadIdx.x;
        float E[4] = {0.f, 0.f, 0.f, 0.f}, I[4] = {0.f, 0.f, 0.f, 0.f};
        if (r4 + 4 <= total) {
            const float4 e4 = *reinterpret_cast<const float4*>(a.Eb + r4);
            const float4 i4 = *reinterpret_cast<const float4*>(a.If + r4);
            E[0] = e4.x; E[1] = e4.y; E[2] = e4.z; E[3] = e4.w;
            I[0] = i4.x; I[1] = i4.y; I[2] = i4.z; I[3] = i4.w;
        } else {
            for (int j = 0; j < 4; j++)
                if (r4 + j < total) {
                    E[j] = a.Eb[r4 + j];
                    I[j] = a.If[r4 + j];
                }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int st = 0;
            if (r4 + j < total && refine_take(a, r4 + j, E[j], I[j], st)) {
                const int slot = atomicAdd(&sn, 1);
                sr[slot] = r4 + j;
                ss[slot] = st;
            }
        }
        __syncthreads();
        if (sn > kSelCap - kChunk) flush();  // uniform: every thread reads sn after the barrier
    }
    __syncthreads();
    flush();
}

// Evaluation: every warp of a persistent grid takes candidates from the list
// (a stride of the grid's warp count) and re-evaluates them.
__global__ void __launch_bounds__(kRefThreads) k_refine_eval(const RefineArgs a)
{
    pdl_enter();
    __shared__ float4 ssc[256];
    __shared__ float2 sex[64];
    if (*a.abort_flag) return;
    const long long total = (long long)*a.nref;
    if (total == 0) return;
    for (int i = threadIdx.x; i < 256; i += kRefThreads) ssc[i] = a.sc[i];
    if (threadIdx.x < 64) sex[threadIdx.x] = a.ex[threadIdx.x];
    __syncthreads();
    const long long nw = (long long)gridDim.x * kRefWarps;
    for (long long i = (long long)blockIdx.x * kRefWarps + (threadIdx.x >> 5); i < total; i += nw)
        refine_one(a, a.cand_r[i], a.cand_s[i], ssc, sex);
}

void launch_refine(const RefineArgs& a, cudaStream_t st, bool pdl)
{
    if (a.n_struct <= 0) return;
    static int per_sm_cache[64][2] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int per_sel = (dev >= 0 && dev < 64) ? per_sm_cache[dev][0] : 0, per_ev = (dev >= 0 && dev < 64) ? per_sm_cache[dev][1] : 0;
    if (per_sel < 1 || per_ev < 1) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sel, k_refine_select, kRefThreads, 0) != cudaSuccess ||
            per_sel < 1)
            per_sel = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_ev, k_refine_eval, kRefThreads, 0) != cudaSuccess ||
            per_ev < 1)
            per_ev = 1;
        if (dev >= 0 && dev < 64) {
            per_sm_cache[dev][0] = per_sel;
            per_sm_cache[dev][1] = per_ev;
        }
    }
    // grid-stride selection over the reflections; the evaluation grid is persistent
    if (pdl) launch_pdl(k_refine_select, a.grid * per_sel, kRefThreads, 0, st, a);
    else k_refine_select<<<a.grid * per_sel, kRefThreads, 0, st>>>(a);
    launch_pdl(k_refine_eval, a.grid * per_ev, kRefThreads, 0, st, a);
}

}  // namespace xrd
