// Steps S4-S6 for the largest size class (structures above 6144 reflections):
// sort by 2-theta, anchor merge, families, cutoff and scaling (Sec. 2, Sec. 3)
// as flat passes over all of the class's reflections at once.
//
// One CTA per structure (on global scratch, beyond shared memory) would leave
// most SMs idle when a few structures hold most of the reflections (256 cells of 20 000-190 000
// reflections, or the single 50 A cell of Sec. 4.2 with 680 000). Here the
// class's structures are laid end to end in one virtual index space (virtual
// offsets voff[j] in class-list order), every step is a loop over that space
// (each CTA one contiguous block of it, its threads following their structure
// forward; the scatter strides over the whole grid instead), and the
// per-structure block steps become device-wide ones:
//  1. bucket of every reflection on |g|^3 (n_j buckets for a structure of n_j
//     reflections, laid out from voff[j] like its reflections), counts by
//     atomics;
//  2. one exclusive scan over all buckets: since a structure's buckets hold
//     exactly its n_j reflections, bucket starts are sorted positions;
//  3. scatter of 16-byte (|g|^2, key, I) records into bucket order, then each
//     bucket sorted in place on the full key (|g|^2, then -h, -k, -l): every
//     later pass reads the sorted records sequentially instead of through a
//     permutation;
//  4. the anchor merge: a definite start where the gap to the previous
//     reflection is >= tol, one thread per run of close reflections;
//  5. a scan of the peak starts gives peak ids; per peak the merged intensity,
//     the family count, and the structure's largest peak (atomic maximum);
//  6. one scan of kept peaks and of their families; per kept peak the staging
//     of the outputs, as the one-CTA kernel writes them.
// The decisions and the order of every floating-point operation are those of
// the one-CTA kernel (k_post.cu), so the outputs are identical. All steps run
// in one cooperative launch separated by grid-wide barriers; a scan is two
// steps (segment sums, then segments offset by the sums before them) over a
// length read from device memory, so the launch is fixed and capturable.
#include "xrd_internal.cuh"
#include "xrd_launch.h"
#include "xrd_post.cuh"

namespace xrd {

constexpr int kPfThreads = 1024;
constexpr int kPfCtasPerSm = 2;  // 64 warps per SM for the latency-bound passes (32 registers a thread)
constexpr unsigned long long kPfWaitNs = 1000000000ull;  // grid barrier time limit: 1 s

__device__ __forceinline__ unsigned long long pf_now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of the cooperative launch (every CTA is resident). bar[0]
// counts arrivals, bar[1] is the generation, bar[2] the failure word; all three
// are zero at the start of a batch. The last CTA to arrive clears the count and
// advances the generation; the others wait for the generation to move, for at
// most kPfWaitNs, or until a failure is posted. Returns false (every CTA, within
// the time limit) once any wait has run out. `extra` arrivals that never come
// (a test of the bounded wait; 0 otherwise) make every wait run out.
__device__ bool pf_grid_sync(int* bar, int G, int extra)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int* vb = bar;
        int good = vb[2] == 0;
        if (good) {
            const int gen = vb[1];
            __threadfence();
            if (atomicAdd(&bar[0], 1) == G - 1 + extra) {
                atomicExch(&bar[0], 0);
                __threadfence();
                atomicAdd(&bar[1], 1);
            } else {
                const unsigned long long t0 = pf_now_ns();
                while (vb[1] == gen) {
                    if (vb[2] != 0 || pf_now_ns() - t0 > kPfWaitNs) {
                        atomicExch(&bar[2], 1);
                        good = 0;
                        break;
                    }
                    __nanosleep(128);
                }
            }
            __threadfence();
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// largest j in [0, c5) with voff[j] <= v (voff[c5] > v)
__device__ __forceinline__ int vowner(const int* __restrict__ voff, int c5, int v)
{
    int lo = 0, hi = c5;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (voff[mid] <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int2 warp_incl_scan2(int2 v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, v.x, o), y = __shfl_up_sync(0xffffffffu, v.y, o);
        if (lane >= o) {
            v.x += x;
            v.y += y;
        }
    }
    return v;
}

// Exclusive block scan of one int2 per thread; returns the block total. tmp: 66 ints.
__device__ __forceinline__ int2 block_scan_int2(int2 v, int2& excl, int* tmp)
{
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 inc = warp_incl_scan2(v);
    if (lane == 31) {
        tmp[w] = inc.x;
        tmp[33 + w] = inc.y;
    }
    __syncthreads();
    if (w == 0) {
        const int2 sv = make_int2(lane < nw ? tmp[lane] : 0, lane < nw ? tmp[33 + lane] : 0);
        const int2 si = warp_incl_scan2(sv);
        if (lane < nw) {
            tmp[lane] = si.x - sv.x;
            tmp[33 + lane] = si.y - sv.y;
        }
        if (lane == 31) {
            tmp[32] = si.x;
            tmp[65] = si.y;
        }
    }
    __syncthreads();
    excl = make_int2(tmp[w] + inc.x - v.x, tmp[33 + w] + inc.y - v.y);
    const int2 tot = make_int2(tmp[32], tmp[65]);
    __syncthreads();  // tmp is free again
    return tot;
}

// ---- the three scanned sequences ----
struct SrcBkt {  // bucket counts -> bucket starts, in place; length V
    static __device__ int len(const PostArgs& a) { return a.pf_scal[0]; }
    static __device__ int2 load(const PostArgs& a, int i) { return make_int2(a.g_bkt[i], 0); }
    static __device__ void store(const PostArgs& a, int i, int2 e) { a.g_bkt[i] = e.x; }
    static __device__ void total(const PostArgs& a, int n, int2 t) { a.g_bkt[n] = t.x; }
};
struct SrcPst {  // peak starts -> peak ids, in place; length V; the peak count into pf_scal[1]
    static __device__ int len(const PostArgs& a) { return a.pf_scal[0]; }
    static __device__ int2 load(const PostArgs& a, int i) { return make_int2(a.pf_pst[i], 0); }
    static __device__ void store(const PostArgs& a, int i, int2 e) { a.pf_pst[i] = e.x; }
    static __device__ void total(const PostArgs& a, int n, int2 t)
    {
        a.pf_pst[n] = t.x;
        a.pf_scal[1] = t.x;
    }
};
template <bool FI>
struct SrcKeep {  // per peak (kept, its families if kept) -> kidx, fidx; length = the peak count
    static __device__ int len(const PostArgs& a) { return a.pf_scal[1]; }
    static __device__ int2 load(const PostArgs& a, int k)
    {
        const unsigned long long m = a.pf_smax[a.pf_pj[k]];
        bool keep;
        if (FI) {
            const float imaxf = __uint_as_float((uint32_t)m);
            keep = a.cutoff == 0.0 ||
                   __float_as_uint(((const float*)a.g_psum)[k]) > __float_as_uint((float)a.cutoff * imaxf);
        } else {
            const double imax = __longlong_as_double((long long)m);
            keep = a.cutoff == 0.0 || dbits(a.g_psum[k]) > dbits(a.cutoff * imax);
        }
        return make_int2(keep ? 1 : 0, keep ? a.g_fcnt[k] : 0);
    }
    static __device__ void store(const PostArgs& a, int k, int2 e)
    {
        a.pf_kidx[k] = e.x;
        a.pf_fidx[k] = e.y;
    }
    static __device__ void total(const PostArgs& a, int n, int2 t)
    {
        a.pf_kidx[n] = t.x;
        a.pf_fidx[n] = t.y;
    }
};

// Segment sums: block b takes [b seg, (b + 1) seg) of [0, len).
template <class S>
__device__ void pf_scan_parts(const PostArgs& a, int B, int G)
{
    __shared__ int tmp[66];
    const int n = S::len(a);
    const int seg = (n + G - 1) / G;
    const int lo = min((int)B * seg, n), hi = min(lo + seg, n);
    int2 s = make_int2(0, 0);
    for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
        const int2 v = S::load(a, i);
        s.x += v.x;
        s.y += v.y;
    }
    int2 e;
    const int2 t = block_scan_int2(s, e, tmp);
    if (threadIdx.x == 0) {
        a.pf_parts[B] = t.x;
        a.pf_parts[G + B] = t.y;
    }
}

// Each segment scanned in chunks of blockDim, offset by the sums of the segments before it.
template <class S>
__device__ void pf_scan_final(const PostArgs& a, int B, int G)
{
    __shared__ int tmp[66];
    const int n = S::len(a);
    const int seg = (n + G - 1) / G;
    const int lo = min((int)B * seg, n), hi = min(lo + seg, n);
    int2 carry = make_int2(0, 0), all = make_int2(0, 0);
    for (int b = threadIdx.x; b < G; b += blockDim.x) {  // the sums of the segments before this one, and of all
        const int x = (int)a.pf_parts[b], y = (int)a.pf_parts[G + b];
        if (b < (int)B) {
            carry.x += x;
            carry.y += y;
        }
        all.x += x;
        all.y += y;
    }
    int2 e;
    carry = block_scan_int2(carry, e, tmp);
    all = block_scan_int2(all, e, tmp);
    for (int c0 = lo; c0 < hi; c0 += blockDim.x) {
        const int i = c0 + (int)threadIdx.x;
        const int2 v = i < hi ? S::load(a, i) : make_int2(0, 0);
        int2 e;
        const int2 t = block_scan_int2(v, e, tmp);
        if (i < hi) S::store(a, i, make_int2(carry.x + e.x, carry.y + e.y));
        carry.x += t.x;
        carry.y += t.y;
    }
    if (B == 0 && threadIdx.x == 0) S::total(a, n, all);
}

// Prologue: the virtual offsets of the class's structures (a structure with an
// invalid atom gets none and reports XRD_EINVAL), the structure maxima cleared;
// every block clears the bucket counts over [0, V).
__device__ void pf_prep(const PostArgs& a, int cls, int B, int G)
{
    __shared__ int tmp[66];
    const int c5 = a.cls_cnt[cls];
    const int* __restrict__ list = a.cls_list + (int64_t)cls * a.n_struct;
    int carry = 0;
    for (int c0 = 0; c0 < c5; c0 += blockDim.x) {
        const int j = c0 + (int)threadIdx.x;
        int nj = 0;
        if (j < c5) {
            const int s = list[j];
            const bool bad = a.atom_bad && a.atom_bad[s];
            nj = bad ? 0 : (int)(a.refl_off[s + 1] - a.refl_off[s]);
            if (B == 0) {
                a.pf_smax[j] = 0ull;
                if (bad) {
                    a.npk[s] = 0;
                    a.nfm[s] = 0;
                    if (a.status[s] == XRD_OK) {
                        a.status[s] = XRD_EINVAL;
                        atomicAdd((unsigned long long*)&a.totals[3], 1ull);
                    }
                }
            }
        }
        int2 e;
        const int2 t = block_scan_int2(make_int2(nj, 0), e, tmp);
        if (B == 0 && j < c5) a.pf_voff[j] = carry + e.x;
        carry += t.x;
    }
    if (B == 0 && threadIdx.x == 0) {
        a.pf_voff[c5] = carry;
        a.pf_scal[0] = carry;
    }
    for (int i = (int)(B * blockDim.x + threadIdx.x); i < carry; i += (int)(G * blockDim.x))
        a.g_bkt[i] = 0;
}

// Virtual bucket of reflection v of class-list structure j (first = voff[j]):
// n_j buckets in |g|^3 over [r2min^1.5, r2max^1.5]
__device__ __forceinline__ int pf_bucket_of(const PostArgs& a, float scale_inv, double q, int first, int nb)
{
    const float qf = d2f_pos(q);
    int b = (int)((qf * sqrtf(qf) - a.lo3) * ((float)nb * scale_inv));
    return first + min(max(b, 0), nb - 1);
}

// The element passes give each CTA one contiguous block of the index space
// [0, len); its threads step through it by blockDim, so a thread's indices
// rise and its structure changes rarely (a structure spans >= 6144 indices).
__device__ __forceinline__ void pf_block(int len, int B, int G, int& lo, int& hi)
{
    const int per = (len + G - 1) / G;
    lo = min(B * per, len);
    hi = min(lo + per, len);
}

// The class-list structure that owns virtual index v, followed forward:
// one bisection for a thread's first index, then a step past each end.
struct PfOwner {
    int j = -1, first = 0, end = 0;
    int64_t rb = 0;  // reflection offset of the structure
    __device__ __forceinline__ void at(const PostArgs& a, const int* __restrict__ list, int c5, int v)
    {
        if (j >= 0 && v < end) return;
        j = j < 0 ? vowner(a.pf_voff, c5, v) : j + 1;
        while (a.pf_voff[j + 1] <= v) j++;
        first = a.pf_voff[j];
        end = a.pf_voff[j + 1];
        rb = a.refl_off[list[j]];
    }
};

// 1. bucket counts
__device__ void pf_bucket(const PostArgs& a, int cls, int B, int G)
{
    const int V = a.pf_scal[0], c5 = a.cls_cnt[cls];
    const int* __restrict__ list = a.cls_list + (int64_t)cls * a.n_struct;
    const float scale_inv = 1.f / (a.hi3 - a.lo3);
    int lo, hi;
    pf_block(V, B, G, lo, hi);
    PfOwner w;
    for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) {
        w.at(a, list, c5, v);
        atomicAdd(&a.g_bkt[pf_bucket_of(a, scale_inv, a.q[w.rb + (v - w.first)], w.first, w.end - w.first)], 1);
    }
}

// 3a. scatter of each reflection's 16-byte record into bucket order (the bucket
// is formed again, by the same arithmetic); g_bkt ends as the bucket ends.
// Grid-stride, unlike the other passes: the whole grid works on the same one or
// two structures at a time, so that their bucket starts (returning atomics)
// and their records (scattered 16-byte stores) stay in L2.
template <bool FI>
__device__ void pf_scatter(const PostArgs& a, int cls, int B, int G)
{
    const int V = a.pf_scal[0], c5 = a.cls_cnt[cls];
    const int* __restrict__ list = a.cls_list + (int64_t)cls * a.n_struct;
    const float scale_inv = 1.f / (a.hi3 - a.lo3);
    PfOwner w;
    for (int v = B * blockDim.x + threadIdx.x; v < V; v += G * blockDim.x) {
        if (v >= w.end) w.j = -1;  // a stride crosses structures: bisect again
        w.at(a, list, c5, v);
        const int64_t r = w.rb + (v - w.first);
        PfRec rec;
        rec.q = a.q[r];
        rec.key = a.key[r];
        rec.I = FI ? a.If[r] : 0.f;
        const int pos = atomicAdd(&a.g_bkt[pf_bucket_of(a, scale_inv, rec.q, w.first, w.end - w.first)], 1);
        a.pf_rec[pos] = rec;
        if (!FI) a.pf_rI[pos] = a.I[r];
    }
}

// 3b. each bucket sorted in place on the full key (|g|^2, then -h, -k, -l) by
// one thread: buckets hold about one reflection on average, so an insertion
// sort over the bucket's few contiguous records
template <bool FI>
__device__ void pf_sortb(const PostArgs& a, int B, int G)
{
    const int V = a.pf_scal[0];
    PfRec* __restrict__ rec = a.pf_rec;
    int lo, hi;
    pf_block(V, B, G, lo, hi);
    for (int vb = lo + threadIdx.x; vb < hi; vb += blockDim.x) {
        const int b0 = vb ? a.g_bkt[vb - 1] : 0, b1 = a.g_bkt[vb];
        for (int i = b0 + 1; i < b1; i++) {
            const PfRec x = rec[i];
            const double xI = FI ? 0.0 : a.pf_rI[i];
            int j = i - 1;
            for (; j >= b0; j--) {
                const PfRec y = rec[j];
                if (!before(x.q, x.key, y.q, y.key)) break;
                rec[j + 1] = y;
                if (!FI) a.pf_rI[j + 1] = a.pf_rI[j];
            }
            if (j + 1 != i) {
                rec[j + 1] = x;
                if (!FI) a.pf_rI[j + 1] = xI;
            }
        }
    }
}

// 3c. with a caller's point group: the family key of every sorted record
__device__ void pf_pgkeys(const PostArgs& a, int B, int G)
{
    const int V = a.pf_scal[0];
    int lo, hi;
    pf_block(V, B, G, lo, hi);
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) a.pf_sfk[p] = pg_family_key(a.pf_rec[p].key, a.pg, a.npg);
}

// 4. anchor merge (and the caller's per-reflection list in merge order): pf_pst
// and g_flag mark the peak starts
template <bool FI>
__device__ void pf_merge(const PostArgs& a, int cls, int B, int G)
{
    const int V = a.pf_scal[0], c5 = a.cls_cnt[cls];
    const int* __restrict__ list = a.cls_list + (int64_t)cls * a.n_struct;
    const float l2 = a.l2f, lh = a.lhf, ttol = a.ttol;
    const double lam = a.lambda, tol = a.tol;
    const PfRec* __restrict__ rec = a.pf_rec;
    int lo, hi;
    pf_block(V, B, G, lo, hi);
    PfOwner w;
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) {
        w.at(a, list, c5, p);
        const double qv = rec[p].q;
        if (a.refl_hkl) {
            if (w.rb + (w.end - w.first) <= a.cap_refl) {
                const int64_t o = w.rb + (p - w.first);
                const uint32_t kv = rec[p].key;
                a.refl_hkl[3 * o] = hkl_h(kv);
                a.refl_hkl[3 * o + 1] = hkl_k(kv);
                a.refl_hkl[3 * o + 2] = hkl_l(kv);
                a.refl_tt[o] = two_theta_q(qv, a.l2h, a.l2l, a.ttab);
                a.refl_I[o] = FI ? (double)rec[p].I : a.pf_rI[p];
            }
        }
        const bool start = p == w.first || !tt_close(rec[p - 1].q, qv, l2, lh, ttol, lam, tol);
        if (!start) continue;  // written by the thread of its run's definite start
        a.pf_pst[p] = 1;
        a.g_flag[p] = 1;
        double qa = qv, qprev = qv;
        for (int i = p + 1; i < w.end; i++) {
            const double qi = rec[i].q;
            if (!tt_close(qprev, qi, l2, lh, ttol, lam, tol)) break;  // the next definite start
            qprev = qi;
            const int ps = tt_close(qa, qi, l2, lh, ttol, lam, tol) ? 0 : 1;
            if (ps) qa = qi;
            a.pf_pst[i] = ps;
            a.g_flag[i] = (uint8_t)ps;
        }
    }
}

// 5. per peak: start position, structure, merged intensity, family count; the
// structure's largest peak sum (bits of a non-negative float or double). The
// lanes of a warp take consecutive positions; when they all lie in one
// structure (the common case) the warp combines its maxima first and one lane
// updates the structure's slot, so the slot sees one atomic per warp, not one
// per peak.
template <bool FI>
__device__ void pf_peaks(const PostArgs& a, int cls, int B, int G)
{
    const int V = a.pf_scal[0], c5 = a.cls_cnt[cls];
    const int* __restrict__ list = a.cls_list + (int64_t)cls * a.n_struct;
    const int lane = threadIdx.x & 31;
    const PfRec* __restrict__ rec = a.pf_rec;
    int lo, hi;
    pf_block(V, B, G, lo, hi);
    PfOwner w;
    bool hex = false;
    for (int p0 = lo + (threadIdx.x & ~31); p0 < hi; p0 += blockDim.x) {  // warp-uniform
        const int p = p0 + lane;
        unsigned long long bits = 0ull;
        int j = -1;
        if (p < hi && a.g_flag[p]) {
            if (w.j < 0 || p >= w.end) {
                w.at(a, list, c5, p);
                hex = a.geo[list[w.j]].hex != 0;
            }
            j = w.j;
            const int k = a.pf_pst[p];
            int e = p + 1;
            while (e < w.end && !a.g_flag[e]) e++;
            a.g_pstart[k] = p;
            a.pf_pj[k] = j;
            if (FI) {
                float sum = 2.f * rec[p].I;
                for (int i = p + 1; i < e; i++) sum = fmaf(2.f, rec[i].I, sum);
                ((float*)a.g_psum)[k] = sum;
                bits = __float_as_uint(sum);
            } else {
                double sum = 0.0;
                for (int i = p; i < e; i++) sum += 2.0 * a.pf_rI[i];
                a.g_psum[k] = sum;
                bits = dbits(sum);
            }
            int nfam = 1;
            if (e - p > 1) {  // distinct family keys among the members
                auto fk = [&](int i) -> unsigned long long {
                    return a.pf_sfk ? a.pf_sfk[i] : family_key(rec[i].key, hex);
                };
                nfam = count_families(fk, p, e);
            }
            a.g_fcnt[k] = nfam;
        }
        const unsigned act = __ballot_sync(0xffffffffu, j >= 0);
        if (!act) continue;
        const int j0 = __shfl_sync(0xffffffffu, j, __ffs(act) - 1);
        if (__all_sync(0xffffffffu, j < 0 || j == j0)) {  // one structure: combine, then one atomic
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, o));
            if (lane == 0) {
                unsigned long long* mx = a.pf_smax + j0;
                if (bits > *(volatile unsigned long long*)mx) atomicMax(mx, bits);
            }
        } else if (j >= 0) {
            unsigned long long* mx = a.pf_smax + j;
            if (bits > *(volatile unsigned long long*)mx) atomicMax(mx, bits);
        }
    }
}

// 6. staging of kept peaks and their families at the structure's reflection
// offset, and its kept-peak and family counts. The structure's peaks are
// contiguous in k, so its constants are read once per thread and structure.
template <bool FI>
__device__ void pf_stage(const PostArgs& a, int cls, int B, int G)
{
    const int NP = a.pf_scal[1];
    const int* __restrict__ list = a.cls_list + (int64_t)cls * a.n_struct;
    const PfRec* __restrict__ rec = a.pf_rec;
    int lo, hi;
    pf_block(NP, B, G, lo, hi);
    int j = -1, s = 0, end = 0, k0 = 0, k1 = 0, kb = 0, fb = 0;
    int64_t rb = 0;
    bool hex = false;
    double imax = 0.0, inv_imax = 0.0;
    float imaxf = 0.f, inv_imaxf = 0.f;
    for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) {
        if (j < 0 || k >= k1) {  // the structure of peak k: [k0, k1) are its peaks
            j = a.pf_pj[k];
            s = list[j];
            const int first = a.pf_voff[j];
            end = a.pf_voff[j + 1];
            k0 = a.pf_pst[first];
            k1 = a.pf_pst[end];
            kb = a.pf_kidx[k0];
            fb = a.pf_fidx[k0];
            rb = a.refl_off[s];
            hex = a.geo[s].hex != 0;
            const unsigned long long m = a.pf_smax[j];
            if (FI) {
                imaxf = __uint_as_float((uint32_t)m);
                inv_imaxf = imaxf > 0.f ? 1.f / imaxf : 0.f;
            } else {
                imax = __longlong_as_double((long long)m);
                inv_imax = imax > 0.0 ? 1.0 / imax : 0.0;
            }
        }
        if (k == k0) {
            a.npk[s] = a.pf_kidx[k1] - kb;
            a.nfm[s] = a.pf_fidx[k1] - fb;
        }
        const int ki = a.pf_kidx[k];
        if (a.pf_kidx[k + 1] == ki) continue;  // below the cutoff
        const int i0 = a.g_pstart[k];
        int i1 = i0 + 1;
        while (i1 < end && !a.g_flag[i1]) i1++;
        const int64_t o = rb + (ki - kb);
        a.st_q[o] = rec[i0].q;
        if (FI) {
            const float ps = ((const float*)a.g_psum)[k];
            ((float*)a.st_I)[o] = (a.scaled && imaxf > 0.f) ? (ps == imaxf ? 100.f : 100.f * (ps * inv_imaxf)) : ps;
        } else {
            const double ps = a.g_psum[k];
            a.st_I[o] = (a.scaled && imax > 0.0) ? (ps == imax ? 100.0 : 100.0 * (ps * inv_imax)) : ps;
        }
        const int fo0 = a.pf_fidx[k] - fb;
        a.st_foff[o] = fo0;
        if (i1 - i0 == 1) {
            const int64_t fo = rb + fo0;
            a.st_key[fo] = rec[i0].key;
            a.st_mult[fo] = 2;
            continue;
        }
        auto kf = [&](int i) { return rec[i].key; };
        auto fkf = [&](int i) -> unsigned long long { return a.pf_sfk ? a.pf_sfk[i] : family_key(kf(i), hex); };
        for (int i = i0; i < i1; i++) {  // families, ranked by descending representative
            const unsigned long long fk = fkf(i);
            bool lead = true;
            for (int jj = i0; jj < i && lead; jj++) lead = fkf(jj) != fk;
            if (!lead) continue;
            uint32_t rep = 0;
            int cnt = 0;
            for (int jj = i0; jj < i1; jj++)
                if (fkf(jj) == fk) {
                    rep = max(rep, kf(jj));
                    cnt++;
                }
            int rank = 0;
            for (int mm = i0; mm < i1; mm++) {
                const unsigned long long fm = fkf(mm);
                if (fm == fk) continue;
                bool lm = true;
                for (int jj = i0; jj < mm && lm; jj++) lm = fkf(jj) != fm;
                if (!lm) continue;
                uint32_t rm = 0;
                for (int jj = i0; jj < i1; jj++)
                    if (fkf(jj) == fm) rm = max(rm, kf(jj));
                rank += rm > rep;
            }
            const int64_t fo = rb + fo0 + rank;
            a.st_key[fo] = rep;
            a.st_mult[fo] = 2 * cnt;
        }
    }
}

// A barrier that ran out: the class's structures report XRD_ETIMEOUT and no peaks.
__device__ void pf_fail(const PostArgs& a, int cls, int B, int G)
{
    const int c5 = a.cls_cnt[cls];
    const int* __restrict__ list = a.cls_list + (int64_t)cls * a.n_struct;
    for (int j = B * blockDim.x + threadIdx.x; j < c5; j += G * blockDim.x) {
        const int s = list[j];
        a.npk[s] = 0;
        a.nfm[s] = 0;
        if (atomicExch(&a.status[s], XRD_ETIMEOUT) == XRD_OK) atomicAdd((unsigned long long*)&a.totals[3], 1ull);
    }
}

// All passes in one cooperative launch: the CTAs of the grid are resident at
// once and a grid-wide barrier separates the passes, so a batch without
// structures in this class pays one launch, and a batch with them no launch gaps.
template <bool FI>
__global__ void __launch_bounds__(kPfThreads, kPfCtasPerSm) k_pf_fused(const PostArgs a, int cls)
{
    pdl_enter();
    if (*a.abort_flag) return;  // set before this launch: the same for every CTA
    const int B = blockIdx.x, G = gridDim.x;
    int* bar = a.pf_bar;
    const int extra = a.pf_bar_extra;
#define PF_SYNC()                          \
    if (!pf_grid_sync(bar, G, extra)) {    \
        pf_fail(a, cls, B, G);             \
        return;                            \
    }
    pf_prep(a, cls, B, G);
    PF_SYNC();
    if (a.pf_scal[0] == 0) return;  // no reflection in this class (every CTA reads the same value)
    pf_bucket(a, cls, B, G);
    PF_SYNC();
    pf_scan_parts<SrcBkt>(a, B, G);
    PF_SYNC();
    pf_scan_final<SrcBkt>(a, B, G);
    PF_SYNC();
    pf_scatter<FI>(a, cls, B, G);
    PF_SYNC();
    pf_sortb<FI>(a, B, G);
    PF_SYNC();
    if (a.pf_sfk) {
        pf_pgkeys(a, B, G);
        PF_SYNC();
    }
    pf_merge<FI>(a, cls, B, G);
    PF_SYNC();
    pf_scan_parts<SrcPst>(a, B, G);
    PF_SYNC();
    pf_scan_final<SrcPst>(a, B, G);
    PF_SYNC();
    pf_peaks<FI>(a, cls, B, G);
    PF_SYNC();
    pf_scan_parts<SrcKeep<FI>>(a, B, G);
    PF_SYNC();
    pf_scan_final<SrcKeep<FI>>(a, B, G);
    PF_SYNC();
    pf_stage<FI>(a, cls, B, G);
#undef PF_SYNC
}

template <bool FI>
static void launch_flat_fi(const PostArgs& a, int cls, cudaStream_t st)
{
    // kPfCtasPerSm CTAs per SM (the launch bounds cap the registers so that they fit), or fewer if the
    // occupancy query says so: every CTA of the cooperative grid must be resident
    static int per_sm_cache[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int per_sm = (dev >= 0 && dev < 64) ? per_sm_cache[dev] : 0;
    if (per_sm < 1) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pf_fused<FI>, kPfThreads, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        per_sm = min(per_sm, kPfCtasPerSm);
        if (dev >= 0 && dev < 64) per_sm_cache[dev] = per_sm;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(min(a.grid * per_sm, kPfScanBlocksMax));
    cfg.blockDim = dim3(kPfThreads);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_pf_fused<FI>, a, cls);
}

void launch_post_flat(const PostArgs& a, int cls, cudaStream_t st)
{
    if (a.n_struct <= 0 || !a.pf_voff) return;
    if (a.If) launch_flat_fi<true>(a, cls, st);
    else launch_flat_fi<false>(a, cls, st);
}

}  // namespace xrd
