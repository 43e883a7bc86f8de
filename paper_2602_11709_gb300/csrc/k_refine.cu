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

// largest s in [lo, n) with off[s] <= i, for off[lo] <= i < off[n]
__device__ __forceinline__ int refl_owner(const int64_t* __restrict__ off, int lo, int n, int64_t i)
{
    int hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Selection: every CTA takes one contiguous range of the batch's reflections
// in chunks of 1024, four consecutive reflections per thread. The offsets of
// the structures a chunk can touch are staged in shared memory (a window of
// 128 structures from the chunk's first), so each thread finds its
// structure by bisection there (in global memory only past the window). Flagged
// reflections are appended to the candidate list, one atomic per warp.
constexpr int kRefItems = 4;
constexpr int kRefChunk = kRefThreads * kRefItems;
constexpr int kRefWindow = 128;

__global__ void __launch_bounds__(kRefThreads) k_refine_select(const RefineArgs a)
{
    pdl_enter();
    __shared__ int64_t woff[kRefWindow + 1];
    __shared__ int s_cur;
    if (*a.abort_flag) return;
    const int n = a.n_struct;
    const int64_t total = a.refl_off[n];
    const int64_t nch = (total + kRefChunk - 1) / kRefChunk;
    const int64_t per = (nch + gridDim.x - 1) / gridDim.x;
    const int64_t c_begin = (int64_t)blockIdx.x * per, c_end = min(c_begin + per, nch);
    if (c_begin >= c_end) return;
    if (threadIdx.x == 0) s_cur = refl_owner(a.refl_off, 0, n, c_begin * kRefChunk);
    const int lane = threadIdx.x & 31;
    for (int64_t c = c_begin; c < c_end; c++) {
        const int64_t r0 = c * kRefChunk;
        __syncthreads();  // s_cur is set; the previous chunk is done with the window
        const int sb = s_cur;
        for (int i = threadIdx.x; i <= kRefWindow; i += kRefThreads) woff[i] = a.refl_off[min(sb + i, n)];
        __syncthreads();
        const int64_t rt = r0 + (int64_t)kRefItems * threadIdx.x;  // this thread's first reflection
        int k = 0;  // largest k < kRefWindow with woff[k] <= rt, if the window reaches rt
        int s;
        if (rt < woff[kRefWindow]) {
            int lo = 0, hi = kRefWindow;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (woff[mid] <= rt) lo = mid;
                else hi = mid;
            }
            k = lo;
            s = sb + k;
        } else {
            s = rt < total ? refl_owner(a.refl_off, min(sb + kRefWindow, n - 1), n, rt) : n - 1;
        }
        if (threadIdx.x == kRefThreads - 1) {  // next chunk's first structure: this thread's last reflection's
            int sl = s;
            const int64_t rl = min(rt + kRefItems, total) - 1;
            while (sl + 1 < n && a.refl_off[sl + 1] <= rl) sl++;
            s_cur = sl;
        }
        int64_t cr[kRefItems];
        int cs[kRefItems];
        int nf = 0;
#pragma unroll
        for (int u = 0; u < kRefItems; u++) {
            const int64_t r = rt + u;
            if (r >= total) break;
            while (a.refl_off[s + 1] <= r) s++;  // at most a few steps: four consecutive reflections
            const float I = a.If[r], E = a.Eb[r];
            const float floorI = a.cref * __uint_as_float(a.imax[s]);
            const bool bad = a.atom_bad && a.atom_bad[s];
            if (!bad && E > 0.f && E > a.tau * fmaxf(I, floorI)) {
                cr[nf] = r;
                cs[nf] = s;
                nf++;
            }
        }
        // append: one atomic per warp
        const int incl = warp_incl_scan(nf);
        const int wtot = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0;
        if (lane == 31 && wtot > 0) base = atomicAdd(a.nref, (unsigned long long)wtot);
        base = __shfl_sync(0xffffffffu, base, 31);
        for (int i = 0; i < nf; i++) {
            const unsigned long long o = base + (unsigned long long)(incl - nf + i);
            a.cand_r[o] = cr[i];
            a.cand_s[o] = cs[i];
        }
    }
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
    // every selection CTA takes a contiguous range of the reflections; the evaluation grid is persistent
    if (pdl) launch_pdl(k_refine_select, a.grid * per_sel, kRefThreads, 0, st, a);
    else k_refine_select<<<a.grid * per_sel, kRefThreads, 0, st>>>(a);
    launch_pdl(k_refine_eval, a.grid * per_ev, kRefThreads, 0, st, a);
}

}  // namespace xrd
