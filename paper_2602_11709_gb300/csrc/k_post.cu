// Steps S4-S6: sort by 2-theta, merge within the tolerance, hkl families,
// intensity cutoff and scaling, then compaction into dense CSR outputs.
//
// Sec. 2: reflections closer in 2-theta than a tolerance are merged into one
// peak, and the equivalent reflections of a peak are grouped into hkl families;
// the optional cutoff (Sec. 2) keeps peaks above
// a fraction of the largest one and Sec. 3 compares intensities on a 0-100 scale.
//
// One CTA per structure of up to 6144 reflections, held in shared memory (the
// larger ones run as the flat passes of k_post_flat.cu). The sort is a bucket
// sort in |g|^3 (reflections are uniform in the volume of the sphere, so
// buckets are nearly equally full); each reflection then takes its rank among
// the members of its own bucket on the full key (|g|^2, then -h, -k, -l), one
// thread per reflection.
// The anchor rule is sequential, so it is split: a reflection whose gap to its
// predecessor is >= tol always opens a peak (a definite start); the short runs
// between definite starts are resolved one thread per run.
#include "xrd_internal.cuh"
#include "xrd_launch.h"
#include "xrd_post.cuh"

namespace xrd {

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ constexpr size_t post_smem_of(size_t c)
{
    // q, key, perm (16 bit), bucket ends, flags, peak starts, peak sums, family counts
    return align16(c * 8) + align16(c * 4) + align16(c * 2) + align16((c + 1) * 4) + align16(c) + align16(c * 4) +
           align16(c * 8) + align16(c * 4);
}

size_t post_smem_bytes(int cap) { return post_smem_of((size_t)cap); }

// CTAs per SM that the shared memory of a class allows (228 KB per SM; about
// 2 KB more per CTA for the static arrays and the per-CTA reservation), at most
// 2048 threads: the launch bounds ask the compiler to fit that many CTAs in the
// register file too.
__host__ __device__ constexpr int post_min_blocks(int cap, int nt)
{
    const int b = (int)((228u * 1024u) / (post_smem_of((size_t)cap) + 2048u));
    const int t = 2048 / nt;
    return b < 1 ? 1 : (b < t ? b : t);
}

static __device__ TTab g_ttab[kTabN + 1];

__global__ void k_ttab_init()
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > kTabN) return;
    const double th = (j * (double)kTabStepDeg) * (kPi / 360.0);
    const double sn = sin(th);
    const double S = sn * sn;
    TTab t;
    t.Sh = (float)S;
    t.Sl = (float)(S - (double)t.Sh);
    t.A = (float)sin(2.0 * th);
    t.Bc = (float)cos(2.0 * th);
    g_ttab[j] = t;
}

const TTab* init_tables(cudaStream_t st)
{
    k_ttab_init<<<(kTabN + 1 + 255) / 256, 256, 0, st>>>();
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_ttab) != cudaSuccess) return nullptr;
    return (const TTab*)p;
}

// The common case of a structure whose sorted reflections are all farther apart
// than the tolerance: every reflection is a peak of one family (g and -g, so
// multiplicity 2), and the merge runs, the peak-start scan and the family
// search are skipped. Same arithmetic and outputs as the general path.
template <typename PermT, bool FI>
__device__ void post_singles(const PostArgs& a, int s, int64_t base, int n, const double* q, const uint32_t* key,
                             const float* Is, const PermT* perm, uint8_t* flag, int* pst, double* psum, int* tmp,
                             double* dtmp)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    double imax = 0.0, inv_imax = 0.0;
    float imaxf = 0.f, inv_imaxf = 0.f;
    unsigned long long lmax = 0;
    for (int p = tid; p < n; p += nt) {
        if (FI) {
            const float v = 2.f * Is[perm[p]];
            ((float*)psum)[p] = v;
            lmax = max(lmax, (unsigned long long)__float_as_uint(v));
        } else {
            const double v = 0.0 + 2.0 * a.I[base + perm[p]];
            psum[p] = v;
            lmax = max(lmax, dbits(v));
        }
    }
    const unsigned long long m = block_max_u64(lmax, (unsigned long long*)dtmp);
    if (FI) {
        imaxf = __uint_as_float((uint32_t)m);
        inv_imaxf = imaxf > 0.f ? 1.f / imaxf : 0.f;
    } else {
        imax = __longlong_as_double((long long)m);
        inv_imax = imax > 0.0 ? 1.0 / imax : 0.0;
    }
    const uint32_t thrf = __float_as_uint((float)a.cutoff * imaxf);
    const unsigned long long thr = dbits(a.cutoff * imax);
    for (int p = tid; p < n; p += nt) {
        const bool keep = a.cutoff == 0.0 || (FI ? __float_as_uint(((float*)psum)[p]) > thrf : dbits(psum[p]) > thr);
        flag[p] = keep;
        pst[p] = keep;
    }
    __syncthreads();
    const int nk = block_excl_scan(pst, n, tmp);
    for (int p = tid; p < n; p += nt) {
        if (!flag[p]) continue;
        const int64_t o = base + pst[p];
        const int v = perm[p];
        a.st_q[o] = q[v];
        if (FI) {
            const float ps = ((const float*)psum)[p];
            ((float*)a.st_I)[o] = (a.scaled && imaxf > 0.f) ? (ps == imaxf ? 100.f : 100.f * (ps * inv_imaxf)) : ps;
        } else {
            const double ps = psum[p];
            a.st_I[o] = (a.scaled && imax > 0.0) ? (ps == imax ? 100.0 : 100.0 * (ps * inv_imax)) : ps;
        }
        a.st_foff[o] = pst[p];  // one family per kept peak
        const uint32_t rep = key[v];
        a.st_key[o] = rep;
        a.st_mult[o] = 2;
    }
    if (tid == 0) {
        a.npk[s] = nk;
        a.nfm[s] = nk;
    }
}

// FI: intensities are FP32 (the FP32 structure-factor variants) and peak sums,
// cutoff and scaling run in FP32; otherwise FP64 throughout.
// Is: the FP32 intensities of the structure (shared or global memory).
template <typename PermT, bool FI>
__device__ void post_structure(const PostArgs& a, int s, int64_t base, int n, const double* q, const uint32_t* key,
                               const float* Is, PermT* perm, int* bkt, uint8_t* flag, int* pst, double* psum,
                               int* fcnt, int* tmp, double* dtmp)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const float l2 = a.l2f, lh = a.lhf, ttol = a.ttol;
    const double lam = a.lambda, tol = a.tol;
    const bool hex = a.geo[s].hex != 0;  // Miller-Bravais families
    // family key of the member at merge position i: the caller's point group (precomputed per
    // reflection), else permutation and sign (Miller-Bravais for a hexagonal cell)
    auto fk = [&](int i) -> unsigned long long {
        return a.fkg ? a.fkg[base + perm[i]] : family_key(key[perm[i]], hex);
    };
    // ---- bucket sort on |g|^3 in [r2min^1.5, r2max^1.5] (a monotone map of |g|^2) ----
    // fcnt holds each reflection's bucket and pst the bucket-ordered reflections
    // until the merge step needs them.
    int* const bid = fcnt;
    int* const perm1 = pst;
    const int nb = n;
    const float lo3 = a.lo3, hi3 = a.hi3;
    const float scale = (float)nb / (hi3 - lo3);
    for (int i = tid; i <= nb; i += nt) bkt[i] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
        const float qf = d2f_pos(q[i]);
        int b = (int)((qf * sqrtf(qf) - lo3) * scale);
        b = min(max(b, 0), nb - 1);
        bid[i] = b;
        atomicAdd(&bkt[b], 1);
    }
    __syncthreads();
    block_excl_scan(bkt, nb, tmp);
    for (int i = tid; i < n; i += nt) perm1[atomicAdd(&bkt[bid[i]], 1)] = i;
    __syncthreads();
    // bkt[b] is now the end of bucket b; rank within the bucket gives the position
    for (int p = tid; p < n; p += nt) {
        const int v = perm1[p];
        const int b = bid[v];
        const int b0 = b ? bkt[b - 1] : 0, b1 = bkt[b];
        int r = b0;
        if (b1 - b0 > 1) {
            const double qv = q[v];
            const uint32_t kv = key[v];
            for (int j = b0; j < b1; j++) {
                const int u = perm1[j];
                r += before(q[u], key[u], qv, kv);  // false for u == v
            }
        }
        perm[r] = (PermT)v;
    }
    __syncthreads();
    // ---- the caller's per-reflection list, in merge order ----
    if (a.refl_hkl && base + n <= a.cap_refl) {
        for (int p = tid; p < n; p += nt) {
            const int v = perm[p];
            const int64_t o = base + p;
            const uint32_t kv = key[v];
            a.refl_hkl[3 * o] = hkl_h(kv);
            a.refl_hkl[3 * o + 1] = hkl_k(kv);
            a.refl_hkl[3 * o + 2] = hkl_l(kv);
            a.refl_tt[o] = two_theta_q(q[v], a.l2h, a.l2l, a.ttab);
            a.refl_I[o] = FI ? (double)Is[v] : a.I[base + v];
        }
    }
    // ---- anchor merge: definite starts, then one thread per run ----
    int close_pair = 0;
    for (int i = tid; i < n; i += nt) {
        const bool start = (i == 0) || !tt_close(q[perm[i - 1]], q[perm[i]], l2, lh, ttol, lam, tol);
        flag[i] = start;
        close_pair |= !start;
    }
    if (!__syncthreads_or(close_pair)) {  // no two reflections within the tolerance: every one is a peak
        post_singles<PermT, FI>(a, s, base, n, q, key, Is, perm, flag, pst, psum, tmp, dtmp);
        return;
    }
    for (int i = tid; i < n; i += nt) {
        if (!flag[i]) continue;
        double qa = q[perm[i]];
        pst[i] = 1;
        for (int j = i + 1; j < n && !flag[j]; j++) {
            const double qj = q[perm[j]];
            if (!tt_close(qa, qj, l2, lh, ttol, lam, tol)) {
                pst[j] = 1;
                qa = qj;
            } else {
                pst[j] = 0;
            }
        }
    }
    __syncthreads();
    // peak starts -> peak ids (exclusive scan); bkt becomes the list of peak start positions
    const int np = block_excl_scan(pst, n, tmp);
    for (int i = tid; i < n; i += nt)
        if ((i + 1 < n ? pst[i + 1] : np) != pst[i]) bkt[pst[i]] = i;
    if (tid == 0) bkt[np] = n;
    __syncthreads();
    // ---- per peak: merged intensity (each half-space reflection stands for g and -g) and family count ----
    // Peak sums are >= 0, so their maximum is taken through the bit patterns.
    double imax = 0.0, inv_imax = 0.0;
    float imaxf = 0.f, inv_imaxf = 0.f;
    if (FI) {
        const float* __restrict__ Ig = Is;
        float* ps = (float*)psum;
        unsigned long long lmax = 0;
        for (int p = tid; p < np; p += nt) {
            const int i0 = bkt[p], i1 = bkt[p + 1];
            float sum = 2.f * Ig[perm[i0]];
            for (int i = i0 + 1; i < i1; i++) sum = fmaf(2.f, Ig[perm[i]], sum);
            ps[p] = sum;
            fcnt[p] = i1 - i0 == 1 ? 1 : count_families(fk, i0, i1);
            lmax = max(lmax, (unsigned long long)__float_as_uint(sum));
        }
        imaxf = __uint_as_float((uint32_t)block_max_u64(lmax, (unsigned long long*)dtmp));
        inv_imaxf = imaxf > 0.f ? 1.f / imaxf : 0.f;
        const uint32_t thr = __float_as_uint((float)a.cutoff * imaxf);
        for (int p = tid; p < np; p += nt) {
            const bool keep = a.cutoff == 0.0 || __float_as_uint(ps[p]) > thr;
            flag[p] = keep;
            pst[p] = keep;
            if (!keep) fcnt[p] = 0;
        }
    } else {
        const double* __restrict__ Ig = a.I + base;
        unsigned long long lmax = 0;
        for (int p = tid; p < np; p += nt) {
            const int i0 = bkt[p], i1 = bkt[p + 1];
            double sum = 0.0;
            for (int i = i0; i < i1; i++) sum += 2.0 * Ig[perm[i]];
            psum[p] = sum;
            fcnt[p] = i1 - i0 == 1 ? 1 : count_families(fk, i0, i1);
            lmax = max(lmax, dbits(sum));
        }
        imax = __longlong_as_double((long long)block_max_u64(lmax, (unsigned long long*)dtmp));
        const unsigned long long thr = dbits(a.cutoff * imax);
        if (tid == 0) dtmp[0] = imax > 0.0 ? 1.0 / imax : 0.0;
        __syncthreads();
        inv_imax = dtmp[0];
        // ---- cutoff, then compaction offsets of kept peaks and their families ----
        for (int p = tid; p < np; p += nt) {
            const bool keep = a.cutoff == 0.0 || dbits(psum[p]) > thr;
            flag[p] = keep;
            pst[p] = keep;
            if (!keep) fcnt[p] = 0;
        }
    }
    __syncthreads();
    int nk, nf;
    block_excl_scan2(pst, fcnt, np, tmp, nk, nf);
    for (int p = tid; p < np; p += nt) {
        if (!flag[p]) continue;
        const int i0 = bkt[p], i1 = bkt[p + 1];
        const int64_t o = base + pst[p];
        a.st_q[o] = q[perm[i0]];  // anchor |g|^2: 2-theta and d are formed during compaction
        if (FI) {  // the largest peak maps to exactly 100
            const float ps = ((const float*)psum)[p];
            ((float*)a.st_I)[o] = (a.scaled && imaxf > 0.f) ? (ps == imaxf ? 100.f : 100.f * (ps * inv_imaxf)) : ps;
        } else {
            const double ps = psum[p];
            a.st_I[o] = (a.scaled && imax > 0.0) ? (ps == imax ? 100.0 : 100.0 * (ps * inv_imax)) : ps;
        }
        a.st_foff[o] = fcnt[p];
        if (i1 - i0 == 1) {  // one reflection: one family of multiplicity 2 (g and -g)
            const uint32_t rep = key[perm[i0]];
            const int64_t fo = base + fcnt[p];
            a.st_key[fo] = rep;
            a.st_mult[fo] = 2;
            continue;
        }
        // families: leaders are first members of each family; rank by descending representative
        for (int i = i0; i < i1; i++) {
            const unsigned long long fi = fk(i);
            bool lead = true;
            for (int j = i0; j < i && lead; j++) lead = fk(j) != fi;
            if (!lead) continue;
            uint32_t rep = 0;
            int cnt = 0;
            for (int j = i0; j < i1; j++)
                if (fk(j) == fi) { rep = max(rep, key[perm[j]]); cnt++; }
            int rank = 0;
            for (int m = i0; m < i1; m++) {  // other leaders with a larger representative
                const unsigned long long fm = fk(m);
                if (fm == fi) continue;
                bool lm = true;
                for (int j = i0; j < m && lm; j++) lm = fk(j) != fm;
                if (!lm) continue;
                uint32_t rm = 0;
                for (int j = i0; j < i1; j++)
                    if (fk(j) == fm) rm = max(rm, key[perm[j]]);
                rank += rm > rep;
            }
            const int64_t fo = base + fcnt[p] + rank;
            a.st_key[fo] = rep;
            a.st_mult[fo] = 2 * cnt;
        }
    }
    if (tid == 0) {
        a.npk[s] = nk;
        a.nfm[s] = nf;
    }
}

// Persistent CTAs over one size class of structures (a list built by the scan
// kernel, largest first), each CTA claiming the next structure from a counter.
// The structure's reflections live in shared memory (n <= CAP); the FP32
// variants also stage the intensities there, in the second half of the
// peak-sum area (FP32 peak sums use the first half).
template <int CAP, int NT, bool FI>
__global__ void __launch_bounds__(NT, post_min_blocks(CAP, NT)) k_post(const PostArgs a, int cls)
{
    static_assert(CAP > 0, "the largest class runs as the flat passes");
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int tmp[66];
    __shared__ double dtmp[32];
    __shared__ int claim;
    if (*a.abort_flag) return;
    const int cnt = a.cls_cnt[cls];
    const int* __restrict__ list = a.cls_list + (int64_t)cls * a.n_struct;
    for (;;) {
        __syncthreads();  // the previous structure is done with shared memory and claim
        if (threadIdx.x == 0) claim = atomicAdd(a.cls_next + cls, 1);
        __syncthreads();
        const int li = claim;
        if (li >= cnt) break;
        const int s = list[li];
        const int64_t base = a.refl_off[s];
        const int n = (int)(a.refl_off[s + 1] - base);
        if (a.atom_bad && a.atom_bad[s]) {  // an invalid atom: no peaks, the structure reports XRD_EINVAL
            if (threadIdx.x == 0) {
                a.npk[s] = 0;
                a.nfm[s] = 0;
                if (a.status[s] == XRD_OK) {
                    a.status[s] = XRD_EINVAL;
                    atomicAdd((unsigned long long*)&a.totals[3], 1ull);
                }
            }
            continue;
        }
        if (n == 0) {
            if (threadIdx.x == 0) { a.npk[s] = 0; a.nfm[s] = 0; }
            continue;
        }
        {
            const size_t c = (size_t)CAP;
            unsigned char* p = smem;
            double* sq = (double*)p; p += align16(c * 8);
            uint32_t* sk = (uint32_t*)p; p += align16(c * 4);
            uint16_t* perm = (uint16_t*)p; p += align16(c * 2);
            int* bkt = (int*)p; p += align16((c + 1) * 4);
            uint8_t* flag = (uint8_t*)p; p += align16(c);
            int* pst = (int*)p; p += align16(c * 4);
            double* psum = (double*)p; p += align16(c * 8);
            int* fcnt = (int*)p;
            float* sI = (float*)psum + c;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                sq[i] = a.q[base + i];
                sk[i] = a.key[base + i];
                if (FI) sI[i] = a.If[base + i];
            }
            __syncthreads();
            post_structure<uint16_t, FI>(a, s, base, n, sq, sk, sI, perm, bkt, flag, pst, psum, fcnt, tmp, dtmp);
        }
    }
}

// Exclusive scans of kept peaks and families per structure (single block),
// output capacity check, totals. The structures are walked in chunks of
// kOutItems * blockDim: coalesced loads into registers, then a transpose
// through shared memory so that each thread scans consecutive structures.
constexpr int kOutThreads = 1024;
constexpr int kOutItems = 4;

__global__ void __launch_bounds__(kOutThreads) k_scan_out(const CompactArgs a)
{
    pdl_enter();
    __shared__ long long ws[33];
    __shared__ long long buf[kOutItems * kOutThreads];
    if (*a.abort_flag) return;
    const int n = a.n_struct, nt = blockDim.x, tid = threadIdx.x, CH = kOutItems * nt;
    long long cp = 0, cf = 0;
    for (int base = 0; base < n; base += CH) {
        long long vp[kOutItems], vf[kOutItems];
#pragma unroll
        for (int u = 0; u < kOutItems; u++) {
            const int i = base + u * nt + tid;
            vp[u] = i < n ? a.npk[i] : 0;
            vf[u] = i < n ? a.nfm[i] : 0;
        }
        long long tp, tf;
        chunk_scan<kOutItems>(vp, buf, ws, &tp);
        chunk_scan<kOutItems>(vf, buf, ws, &tf);
#pragma unroll
        for (int u = 0; u < kOutItems; u++) {
            const int i = base + u * nt + tid;
            if (i < n) {
                a.out.peak_off[i] = cp + vp[u];
                a.fam_soff[i] = cf + vf[u];
                if (a.out.refl_off) a.out.refl_off[i] = a.refl_off[i];
            }
        }
        cp += tp;
        cf += tf;
    }
    const bool over = cp > a.cap_peaks || cf > a.cap_fam || (a.out.refl_off && a.refl_off[n] > a.out.cap_refl);
    if (over)
        for (int i = tid; i < n; i += nt) a.out.status[i] = XRD_ECAPACITY;
    if (tid == 0) {
        a.out.peak_off[n] = cp;
        a.fam_soff[n] = cf;
        a.out.totals[1] = cp;
        a.out.totals[2] = cf;
        if (a.out.refl_off) a.out.refl_off[n] = a.refl_off[n];
        *a.out_abort = over;
        if (over) a.out.totals[3] = n;
        else a.out.fam_off[cp] = cf;
    }
}

// Multi-block form of k_scan_out for batches of more than two chunks: chunk
// sums of kept peaks and families first, then every chunk scans its own
// structures from the sums of the chunks before it.
__global__ void __launch_bounds__(kOutThreads) k_scan_out_parts(const CompactArgs a)
{
    pdl_enter();
    __shared__ long long ws[33];
    if (*a.abort_flag) return;
    const int n = a.n_struct, nt = blockDim.x, tid = threadIdx.x, base = blockIdx.x * kOutItems * nt;
    long long p = 0, f = 0;
#pragma unroll
    for (int u = 0; u < kOutItems; u++) {
        const int i = base + u * nt + tid;
        if (i < n) {
            p += a.npk[i];
            f += a.nfm[i];
        }
    }
    long long tp, tf;
    block_prefix_ll(p, ws, &tp);
    block_prefix_ll(f, ws, &tf);
    if (tid == 0) {
        a.parts[2 * blockIdx.x] = tp;
        a.parts[2 * blockIdx.x + 1] = tf;
    }
}

__global__ void __launch_bounds__(kOutThreads) k_scan_out_final(const CompactArgs a)
{
    pdl_enter();
    __shared__ long long ws[33];
    __shared__ long long buf[kOutItems * kOutThreads];
    __shared__ long long pre[2], all[2];
    if (*a.abort_flag) return;
    const int n = a.n_struct, nt = blockDim.x, tid = threadIdx.x, b = blockIdx.x, base = b * kOutItems * nt;
    if (tid < 2) {
        long long q = 0, t = 0;
        for (int c = 0; c < (int)gridDim.x; c++) {
            const long long v = a.parts[2 * c + tid];
            q += c < b ? v : 0;
            t += v;
        }
        pre[tid] = q;
        all[tid] = t;
    }
    __syncthreads();
    const long long cp = all[0], cf = all[1];
    const bool over = cp > a.cap_peaks || cf > a.cap_fam || (a.out.refl_off && a.refl_off[n] > a.out.cap_refl);
    long long vp[kOutItems], vf[kOutItems], tp, tf;
#pragma unroll
    for (int u = 0; u < kOutItems; u++) {
        const int i = base + u * nt + tid;
        vp[u] = i < n ? a.npk[i] : 0;
        vf[u] = i < n ? a.nfm[i] : 0;
    }
    chunk_scan<kOutItems>(vp, buf, ws, &tp);
    chunk_scan<kOutItems>(vf, buf, ws, &tf);
#pragma unroll
    for (int u = 0; u < kOutItems; u++) {
        const int i = base + u * nt + tid;
        if (i < n) {
            a.out.peak_off[i] = pre[0] + vp[u];
            a.fam_soff[i] = pre[1] + vf[u];
            if (a.out.refl_off) a.out.refl_off[i] = a.refl_off[i];
            if (over) a.out.status[i] = XRD_ECAPACITY;
        }
    }
    if (b == 0 && tid == 0) {
        if (a.out.refl_off) a.out.refl_off[n] = a.refl_off[n];
        a.out.peak_off[n] = cp;
        a.fam_soff[n] = cf;
        a.out.totals[1] = cp;
        a.out.totals[2] = cf;
        *a.out_abort = over;
        if (over) a.out.totals[3] = n;
        else a.out.fam_off[cp] = cf;
    }
}

// largest s in [lo, n) with off[s] <= i, for off[lo] <= i < off[n]
__device__ __forceinline__ int owner(const int64_t* __restrict__ off, int lo, int n, int64_t i)
{
    int hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Kept peaks and their families into the dense CSR outputs, one thread per
// output peak. Each block takes one contiguous range of output peaks: thread 0
// finds the structure of the range's first peak by bisection, and every
// thread then walks forward from the structure of the previous 256 peaks (a
// few steps; bisection again past eight). 2-theta and d are formed here from
// the anchor |g|^2.
constexpr int kCompactThreads = 256;

__global__ void __launch_bounds__(kCompactThreads) k_compact(const CompactArgs a)
{
    pdl_enter();
    __shared__ int s_cur;
    if (*a.abort_flag || *a.out_abort) return;
    const int n = a.n_struct, tid = threadIdx.x;
    const int64_t* __restrict__ poff = a.out.peak_off;
    const int64_t total = poff[n];
    const int64_t per = ((total + gridDim.x - 1) / gridDim.x + kCompactThreads - 1) / kCompactThreads * kCompactThreads;
    const int64_t start = (int64_t)blockIdx.x * per, end = min(start + per, total);
    if (start >= end) return;
    if (tid == 0) s_cur = owner(poff, 0, n, start);
    __syncthreads();
    for (int64_t P0 = start; P0 < end; P0 += kCompactThreads) {
        const int64_t P = P0 + tid;
        int s = s_cur;
        if (P < end) {
            for (int k = 0; k < 8 && poff[s + 1] <= P; k++) s++;
            if (poff[s + 1] <= P) s = owner(poff, s + 1, n, P);
            const int64_t pe = poff[s + 1];
            const int64_t rb = a.refl_off[s];
            const int64_t src = rb + (P - poff[s]);
            const double qa = a.st_q[src];
            a.out.two_theta[P] = two_theta_q(qa, a.l2h, a.l2l, a.ttab);
            a.out.d_hkl[P] = inv_sqrt_df(qa);
            a.out.intensity[P] = a.fi ? f2d_fast(((const float*)a.st_I)[src]) : a.st_I[src];
            const int64_t fs = a.fam_soff[s];
            const int64_t f0 = fs + a.st_foff[src];
            const int64_t f1 = P + 1 < pe ? fs + a.st_foff[src + 1] : a.fam_soff[s + 1];
            a.out.fam_off[P] = f0;
            for (int64_t F = f0; F < f1; F++) {
                const int64_t fsrc = rb + (F - fs);
                const uint32_t rep = a.st_key[fsrc];
                a.out.hkl[3 * F] = hkl_h(rep);
                a.out.hkl[3 * F + 1] = hkl_k(rep);
                a.out.hkl[3 * F + 2] = hkl_l(rep);
                a.out.mult[F] = a.st_mult[fsrc];
            }
        }
        __syncthreads();  // every thread has read s_cur
        if (tid == kCompactThreads - 1) s_cur = s;  // owner of this pass's last peak
        __syncthreads();
    }
}

template <int CAP, int NT, bool FI>
static void launch_post_class(const PostArgs& a, int cls, cudaStream_t st)
{
    const size_t smem = post_smem_bytes(CAP);
    static int per_sm_cache[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int per_sm = (dev >= 0 && dev < 64) ? per_sm_cache[dev] : 0;
    if (per_sm < 1) {
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_post<CAP, NT, FI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        // all of the unified L1 / shared storage as shared memory: more structures in flight per SM
        cudaFuncSetAttribute(k_post<CAP, NT, FI>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_post<CAP, NT, FI>, NT, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        if (dev >= 0 && dev < 64) per_sm_cache[dev] = per_sm;
    }
    const int grid = min(a.grid * per_sm, a.n_struct);
    k_post<CAP, NT, FI><<<grid, NT, smem, st>>>(a, cls);
}

// st[c]: the stream of size class c (the caller forks and joins them); the largest first
template <bool FI>
static void launch_post_fi(const PostArgs& a, const cudaStream_t* st)
{
    launch_post_flat(a, kPostFlatClass, st[kPostFlatClass]);
    launch_post_class<kPostCap7, 1024, FI>(a, 7, st[7]);
    launch_post_class<kPostCap6, 512, FI>(a, 6, st[6]);
    launch_post_class<kPostCap5, 512, FI>(a, 5, st[5]);
    launch_post_class<kPostCap4, 256, FI>(a, 4, st[4]);
    launch_post_class<kPostCap3, 256, FI>(a, 3, st[3]);
    launch_post_class<kPostCap2, 192, FI>(a, 2, st[2]);
    launch_post_class<kPostCap1, 128, FI>(a, 1, st[1]);
    launch_post_class<kPostCap0, 64, FI>(a, 0, st[0]);
}

// With a caller's point group: the family key of every reflection of the batch
// (once per call; the post kernels then compare keys instead of forming orbits).
__global__ void __launch_bounds__(256) k_pg_keys(const PostArgs a, unsigned long long* __restrict__ fkg)
{
    pdl_enter();
    if (*a.abort_flag) return;
    const int64_t total = a.refl_off[a.n_struct];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x)
        fkg[r] = pg_family_key(a.key[r], a.pg, a.npg);
}

void launch_pg_keys(const PostArgs& a, unsigned long long* fkg, cudaStream_t st)
{
    if (a.n_struct > 0 && fkg) launch_pdl(k_pg_keys, a.grid * 8, 256, 0, st, a, fkg);
}

// a.grid = number of SMs
void launch_post(const PostArgs& a, const cudaStream_t* st)
{
    if (a.n_struct <= 0) return;
    if (a.If) launch_post_fi<true>(a, st);
    else launch_post_fi<false>(a, st);
}

void launch_compact(const CompactArgs& a, cudaStream_t st)
{
    const int nch = (a.n_struct + kOutItems * kOutThreads - 1) / (kOutItems * kOutThreads);
    if (nch <= 2 || !a.parts) {
        k_scan_out<<<1, kOutThreads, 0, st>>>(a);
    } else {
        k_scan_out_parts<<<nch, kOutThreads, 0, st>>>(a);
        launch_pdl(k_scan_out_final, nch, kOutThreads, 0, st, a);
    }
    if (a.n_struct > 0) launch_pdl(k_compact, a.grid * 8, kCompactThreads, 0, st, a);
}

}  // namespace xrd
