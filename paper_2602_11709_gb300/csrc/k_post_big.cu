// Steps S4-S6 for the largest structures: sort by 2-theta, anchor merge,
// families, cutoff and scaling (Sec. 2, Sec. 3), one thread-block cluster per
// structure.
//
// A structure with more reflections than the shared-memory classes hold
// (above 6144) is one 1024-thread CTA working on global scratch; a single
// structure of several hundred thousand reflections (the 50 A, 940-atom cell
// of Sec. 4.2) then kept one SM busy for milliseconds while the others idled.
// Above a threshold (65536 reflections when the class holds few structures,
// 262144 when it holds many: then one CTA per structure keeps every SM busy and
// has more throughput) the CTAs of a cluster (16, or 8, co-scheduled on one
// GPC) share one structure instead: every loop strides over all the cluster's threads, and the
// block-wide steps (bucket scan, the OR of "any close pair", the maximum, the
// scans of peak and family counts) become cluster-wide, combining per-CTA
// partial results through a small per-cluster area of global memory between
// cluster barriers. The arithmetic and the order of every decision are those
// of the one-CTA kernel, so the outputs are identical.
//
// This file is compiled with global loads cached in L2 only (-Xptxas -dlcm=cg):
// data one CTA of the cluster writes is read by the others after a fence and a
// cluster barrier, and must not be served from an SM's own L1.
#include <cooperative_groups.h>

#include "xrd_internal.cuh"
#include "xrd_launch.h"
#include "xrd_post.cuh"

namespace cg = cooperative_groups;

namespace xrd {

constexpr int kBigThreads = 1024;

// The CTAs of one cluster working on one structure.
struct Team {
    int rank, size;   // this CTA's rank in the cluster, the cluster's CTA count
    long long* part;  // the cluster's area: [2 * kPostClusterMax] partial results
    __device__ int gt() const { return rank * kBigThreads + (int)threadIdx.x; }
    __device__ int gn() const { return size * kBigThreads; }
};

__device__ __forceinline__ void team_sync()
{
    __threadfence();            // this CTA's global writes reach L2
    cg::this_cluster().sync();  // every CTA of the cluster arrives, with release/acquire order
}

// Exclusive prefix sum of a[0..n) (global) by the cluster: each CTA scans a
// contiguous segment, then adds the totals of the segments before it. Returns
// the total; ends with the array final and the partial area free again.
__device__ int team_excl_scan(const Team& t, int* a, int n, int* tmp)
{
    const int seg = (n + t.size - 1) / t.size;
    const int lo = min(t.rank * seg, n), hi = min(lo + seg, n);
    const int tot = block_excl_scan(a + lo, hi - lo, tmp);
    if (threadIdx.x == 0) t.part[t.rank] = tot;
    team_sync();
    long long off = 0, all = 0;
    for (int r = 0; r < t.size; r++) {
        const long long v = __ldcg(t.part + r);
        off += r < t.rank ? v : 0;
        all += v;
    }
    for (int i = lo + (int)threadIdx.x; i < hi; i += kBigThreads) a[i] += (int)off;
    team_sync();
    return (int)all;
}

// Two exclusive prefix sums of the same length at once (a and b); totals in ta, tb.
__device__ void team_excl_scan2(const Team& t, int* a, int* b, int n, int* tmp, int& ta, int& tb)
{
    const int seg = (n + t.size - 1) / t.size;
    const int lo = min(t.rank * seg, n), hi = min(lo + seg, n);
    int sa, sb;
    block_excl_scan2(a + lo, b + lo, hi - lo, tmp, sa, sb);
    if (threadIdx.x == 0) {
        t.part[t.rank] = sa;
        t.part[kPostClusterMax + t.rank] = sb;
    }
    team_sync();
    long long oa = 0, ob = 0, aa = 0, ab = 0;
    for (int r = 0; r < t.size; r++) {
        const long long va = __ldcg(t.part + r), vb = __ldcg(t.part + kPostClusterMax + r);
        oa += r < t.rank ? va : 0;
        ob += r < t.rank ? vb : 0;
        aa += va;
        ab += vb;
    }
    for (int i = lo + (int)threadIdx.x; i < hi; i += kBigThreads) {
        a[i] += (int)oa;
        b[i] += (int)ob;
    }
    team_sync();
    ta = (int)aa;
    tb = (int)ab;
}

__device__ unsigned long long team_max_u64(const Team& t, unsigned long long v, unsigned long long* tmp)
{
    const unsigned long long m = block_max_u64(v, tmp);
    if (threadIdx.x == 0) t.part[t.rank] = (long long)m;
    team_sync();
    unsigned long long r = 0;
    for (int k = 0; k < t.size; k++) r = max(r, (unsigned long long)__ldcg(t.part + k));
    team_sync();
    return r;
}

__device__ bool team_or(const Team& t, int v)
{
    const int any = __syncthreads_or(v);
    if (threadIdx.x == 0) t.part[t.rank] = any;
    team_sync();
    long long r = 0;
    for (int k = 0; k < t.size; k++) r |= __ldcg(t.part + k);
    team_sync();
    return r != 0;
}

// FI: FP32 intensities (peak sums, cutoff and scaling in FP32); otherwise FP64.
template <bool FI>
__device__ void post_team(const PostArgs& a, const Team& t, int s, int64_t base, int n, int* tmp, double* dtmp)
{
    const double* q = a.q + base;
    const uint32_t* key = a.key + base;
    const float* Is = FI ? a.If + base : nullptr;
    int* perm = a.g_perm + base;
    int* bkt = a.g_bkt + base + s;
    uint8_t* flag = a.g_flag + base;
    int* pst = a.g_pstart + base;
    double* psum = a.g_psum + base;
    int* fcnt = a.g_fcnt + base;
    const int gt = t.gt(), gn = t.gn();
    const float l2 = a.l2f, lh = a.lhf, ttol = a.ttol;
    const double lam = a.lambda, tol = a.tol;
    const bool hex = a.geo[s].hex != 0;
    // ---- bucket sort on |g|^3 (fcnt holds the buckets, pst the bucket order until the merge) ----
    int* const bid = fcnt;
    int* const perm1 = pst;
    const int nb = n;
    const float lo3 = a.lo3, hi3 = a.hi3;
    const float scale = (float)nb / (hi3 - lo3);
    for (int i = gt; i <= nb; i += gn) bkt[i] = 0;
    team_sync();
    for (int i = gt; i < n; i += gn) {
        const float qf = d2f_pos(q[i]);
        int b = (int)((qf * sqrtf(qf) - lo3) * scale);
        b = min(max(b, 0), nb - 1);
        bid[i] = b;
        atomicAdd(&bkt[b], 1);
    }
    team_sync();
    team_excl_scan(t, bkt, nb, tmp);
    for (int i = gt; i < n; i += gn) perm1[atomicAdd(&bkt[bid[i]], 1)] = i;
    team_sync();
    for (int p = gt; p < n; p += gn) {  // rank within the bucket on the full key
        const int v = perm1[p];
        const int b = bid[v];
        const int b0 = b ? bkt[b - 1] : 0, b1 = bkt[b];
        int r = b0;
        if (b1 - b0 > 1) {
            const double qv = q[v];
            const uint32_t kv = key[v];
            for (int j = b0; j < b1; j++) {
                const int u = perm1[j];
                r += before(q[u], key[u], qv, kv);
            }
        }
        perm[r] = v;
    }
    team_sync();
    if (a.refl_hkl && base + n <= a.cap_refl) {  // the caller's per-reflection list, in merge order
        for (int p = gt; p < n; p += gn) {
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
    for (int i = gt; i < n; i += gn) {
        const bool start = (i == 0) || !tt_close(q[perm[i - 1]], q[perm[i]], l2, lh, ttol, lam, tol);
        flag[i] = start;
        close_pair |= !start;
    }
    const bool any_close = team_or(t, close_pair);
    int np;
    if (any_close) {
        for (int i = gt; i < n; i += gn) {
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
        team_sync();
        np = team_excl_scan(t, pst, n, tmp);
        for (int i = gt; i < n; i += gn)
            if ((i + 1 < n ? pst[i + 1] : np) != pst[i]) bkt[pst[i]] = i;
        if (gt == 0) bkt[np] = n;
    } else {  // every reflection is a peak of one family (g and -g)
        np = n;
        for (int i = gt; i <= n; i += gn) bkt[i] = i;
    }
    team_sync();
    // ---- per peak: merged intensity and family count; the largest; the cutoff ----
    unsigned long long lmax = 0;
    for (int p = gt; p < np; p += gn) {
        const int i0 = bkt[p], i1 = bkt[p + 1];
        if (FI) {
            float sum = 2.f * Is[perm[i0]];
            for (int i = i0 + 1; i < i1; i++) sum = fmaf(2.f, Is[perm[i]], sum);
            ((float*)psum)[p] = sum;
            lmax = max(lmax, (unsigned long long)__float_as_uint(sum));
        } else {
            double sum = 0.0;
            for (int i = i0; i < i1; i++) sum += 2.0 * a.I[base + perm[i]];
            psum[p] = sum;
            lmax = max(lmax, dbits(sum));
        }
        fcnt[p] = i1 - i0 == 1 ? 1 : count_families(key, perm, i0, i1, hex);
    }
    const unsigned long long m = team_max_u64(t, lmax, (unsigned long long*)dtmp);
    double imax = 0.0, inv_imax = 0.0;
    float imaxf = 0.f, inv_imaxf = 0.f;
    if (FI) {
        imaxf = __uint_as_float((uint32_t)m);
        inv_imaxf = imaxf > 0.f ? 1.f / imaxf : 0.f;
    } else {
        imax = __longlong_as_double((long long)m);
        inv_imax = imax > 0.0 ? 1.0 / imax : 0.0;
    }
    const uint32_t thrf = __float_as_uint((float)a.cutoff * imaxf);
    const unsigned long long thr = dbits(a.cutoff * imax);
    for (int p = gt; p < np; p += gn) {
        const bool keep = a.cutoff == 0.0 || (FI ? __float_as_uint(((float*)psum)[p]) > thrf : dbits(psum[p]) > thr);
        flag[p] = keep;
        pst[p] = keep;
        if (!keep) fcnt[p] = 0;
    }
    team_sync();
    int nk, nf;
    team_excl_scan2(t, pst, fcnt, np, tmp, nk, nf);
    // ---- staging of kept peaks and their families ----
    for (int p = gt; p < np; p += gn) {
        if (!flag[p]) continue;
        const int i0 = bkt[p], i1 = bkt[p + 1];
        const int64_t o = base + pst[p];
        a.st_q[o] = q[perm[i0]];
        if (FI) {
            const float ps = ((const float*)psum)[p];
            a.st_I[o] = f2d_fast((a.scaled && imaxf > 0.f) ? (ps == imaxf ? 100.f : 100.f * (ps * inv_imaxf)) : ps);
        } else {
            const double ps = psum[p];
            a.st_I[o] = (a.scaled && imax > 0.0) ? (ps == imax ? 100.0 : 100.0 * (ps * inv_imax)) : ps;
        }
        a.st_foff[o] = fcnt[p];
        if (i1 - i0 == 1) {
            const uint32_t rep = key[perm[i0]];
            const int64_t fo = base + fcnt[p];
            a.st_hkl[3 * fo] = hkl_h(rep);
            a.st_hkl[3 * fo + 1] = hkl_k(rep);
            a.st_hkl[3 * fo + 2] = hkl_l(rep);
            a.st_mult[fo] = 2;
            continue;
        }
        for (int i = i0; i < i1; i++) {  // families, ranked by descending representative
            const unsigned long long fk = family_key(key[perm[i]], hex);
            bool lead = true;
            for (int j = i0; j < i && lead; j++) lead = family_key(key[perm[j]], hex) != fk;
            if (!lead) continue;
            uint32_t rep = 0;
            int cnt = 0;
            for (int j = i0; j < i1; j++)
                if (family_key(key[perm[j]], hex) == fk) { rep = max(rep, key[perm[j]]); cnt++; }
            int rank = 0;
            for (int mm = i0; mm < i1; mm++) {
                const unsigned long long fm = family_key(key[perm[mm]], hex);
                if (fm == fk) continue;
                bool lm = true;
                for (int j = i0; j < mm && lm; j++) lm = family_key(key[perm[j]], hex) != fm;
                if (!lm) continue;
                uint32_t rm = 0;
                for (int j = i0; j < i1; j++)
                    if (family_key(key[perm[j]], hex) == fm) rm = max(rm, key[perm[j]]);
                rank += rm > rep;
            }
            const int64_t fo = base + fcnt[p] + rank;
            a.st_hkl[3 * fo] = hkl_h(rep);
            a.st_hkl[3 * fo + 1] = hkl_k(rep);
            a.st_hkl[3 * fo + 2] = hkl_l(rep);
            a.st_mult[fo] = 2 * cnt;
        }
    }
    if (gt == 0) {
        a.npk[s] = nk;
        a.nfm[s] = nf;
    }
    team_sync();  // the scratch and the partial area are free for the next structure
}

// Persistent clusters: cluster c takes the structures c, c + C, c + 2C, ... of
// the largest class (a list in largest-first order) and works on those above
// big_min reflections, so every CTA of a cluster walks the same structures and
// reaches the same barriers.
template <bool FI>
__global__ void __launch_bounds__(kBigThreads, 1) k_post_big(const PostArgs a, int cls)
{
    __shared__ int tmp[66];
    __shared__ double dtmp[32];
    if (*a.abort_flag) return;  // the same for every CTA
    const cg::cluster_group cl = cg::this_cluster();
    const int size = (int)cl.num_blocks();
    const int cid = (int)blockIdx.x / size, ncl = (int)gridDim.x / size;
    const Team t{(int)cl.block_rank(), size, a.cpart + (int64_t)cid * 2 * kPostClusterMax};
    const int cnt = a.cls_cnt[cls];
    const int big_min = post_big_min(cnt, a.grid);
    const int* __restrict__ list = a.cls_list + (int64_t)cls * a.n_struct;
    for (int li = cid; li < cnt; li += ncl) {
        const int s = list[li];
        const int64_t base = a.refl_off[s];
        const int n = (int)(a.refl_off[s + 1] - base);
        if (n <= big_min) continue;  // the one-CTA kernel's (the same for every CTA of the cluster)
        if (a.atom_bad && a.atom_bad[s]) {  // an invalid atom: no peaks, the structure reports XRD_EINVAL
            if (t.gt() == 0) {
                a.npk[s] = 0;
                a.nfm[s] = 0;
                if (a.status[s] == XRD_OK) {
                    a.status[s] = XRD_EINVAL;
                    atomicAdd((unsigned long long*)&a.totals[3], 1ull);
                }
            }
            continue;
        }
        post_team<FI>(a, t, s, base, n, tmp, dtmp);
    }
}

// Largest cluster the device co-schedules for this kernel (16, else 8); the grid fills the
// GPU with clusters. Returns false when no cluster fits (the caller then uses one CTA per structure).
template <bool FI>
static bool launch_big_fi(const PostArgs& a, int cls, cudaStream_t st)
{
    static int cache[64][2] = {};  // (cluster size, active clusters) per device
    int dev = 0;
    cudaGetDevice(&dev);
    int csize = (dev >= 0 && dev < 64) ? cache[dev][0] : 0, ncl = (dev >= 0 && dev < 64) ? cache[dev][1] : 0;
    if (csize == 0) {
        cudaFuncSetAttribute(k_post_big<FI>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        csize = -1;
        for (int c : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(c * 64);
            cfg.blockDim = dim3(kBigThreads);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = c;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, k_post_big<FI>, &cfg) == cudaSuccess && nc > 0) {
                csize = c;
                ncl = min(nc, kPostClustersMax);
                break;
            }
        }
        cudaGetLastError();  // a refused size leaves no sticky error
        if (dev >= 0 && dev < 64) {
            cache[dev][0] = csize;
            cache[dev][1] = ncl;
        }
    }
    if (csize <= 0) return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize * ncl);
    cfg.blockDim = dim3(kBigThreads);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_post_big<FI>, a, cls) == cudaSuccess;
}

bool launch_post_big(const PostArgs& a, int cls, cudaStream_t st)
{
    if (!a.cpart) return false;
    return a.If ? launch_big_fi<true>(a, cls, st) : launch_big_fi<false>(a, cls, st);
}

}  // namespace xrd
