// Steps S4-S6: sort by 2-theta, merge within the tolerance, hkl families,
// intensity cutoff and scaling, then compaction into dense CSR outputs.
//
// Sec. 2 of the paper lists "pairwise operations for grouping
// symmetry-equivalent reflections" and "the merging of reflections within
// specified angular tolerances"; the optional cutoff (Sec. 2) keeps peaks above
// a fraction of the largest one and Sec. 3 compares intensities on a 0-100 scale.
//
// One CTA per structure. Reflections of structures up to `cap_smem` live in
// shared memory; larger ones use the same code on global scratch (generic
// pointers). The sort is a bucket sort in |g|^3 (reflections are uniform in
// the volume of the sphere, so buckets are nearly equally full) followed by an
// insertion sort of each bucket on the full key (|g|^2, then -h, -k, -l).
// The anchor rule is sequential, so it is split: a reflection whose gap to its
// predecessor is >= tol always opens a peak (a definite start); the short runs
// between definite starts are resolved one thread per run.
#include "xrd_internal.cuh"
#include "xrd_launch.h"

namespace xrd {

constexpr int kPostThreads = 256;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

size_t post_smem_bytes(int cap)
{
    const size_t c = (size_t)cap;
    return align16(c * 8) + align16(c * 4) + align16(c * 8) + align16(c * 4) + align16((c + 1) * 4) +
           align16(c) + align16(c * 4) + align16(c * 8) + align16(c * 4);
}

// family key: |h|, |k|, |l| sorted descending, packed
__device__ __forceinline__ uint32_t family_key(uint32_t key)
{
    int a = abs(hkl_h(key)), b = abs(hkl_k(key)), c = abs(hkl_l(key));
    int t;
    if (b > a) { t = a; a = b; b = t; }
    if (c > b) { t = b; b = c; c = t; }
    if (b > a) { t = a; a = b; b = t; }
    return ((uint32_t)a << 20) | ((uint32_t)b << 10) | (uint32_t)c;
}

// sort order: ascending |g|^2, ties by descending (h, k, l)
__device__ __forceinline__ bool before(double qa, uint32_t ka, double qb, uint32_t kb)
{
    return qa < qb || (qa == qb && ka > kb);
}

__global__ void __launch_bounds__(kPostThreads) k_post(const PostArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int tmp[34];
    __shared__ double dtmp[32];
    if (*a.abort_flag) return;
    const int s = blockIdx.x;
    const int64_t base = a.refl_off[s];
    const int n = (int)(a.refl_off[s + 1] - base);
    const int tid = threadIdx.x, nt = blockDim.x;
    if (n == 0) {
        if (tid == 0) { a.npk[s] = 0; a.nfm[s] = 0; }
        return;
    }
    const double* __restrict__ Ig = a.I + base;
    const double* q;
    const uint32_t* key;
    double* tt;
    int* perm;
    int* bkt;
    uint8_t* flag;
    int* pst;
    double* psum;
    int* fcnt;
    if (n <= a.cap_smem) {
        const size_t c = (size_t)a.cap_smem;
        unsigned char* p = smem;
        double* sq = (double*)p; p += align16(c * 8);
        uint32_t* sk = (uint32_t*)p; p += align16(c * 4);
        tt = (double*)p; p += align16(c * 8);
        perm = (int*)p; p += align16(c * 4);
        bkt = (int*)p; p += align16((c + 1) * 4);
        flag = (uint8_t*)p; p += align16(c);
        pst = (int*)p; p += align16(c * 4);
        psum = (double*)p; p += align16(c * 8);
        fcnt = (int*)p;
        for (int i = tid; i < n; i += nt) {
            sq[i] = a.q[base + i];
            sk[i] = a.key[base + i];
        }
        q = sq;
        key = sk;
    } else {
        q = a.q + base;
        key = a.key + base;
        tt = a.g_tt + base;
        perm = a.g_perm + base;
        bkt = a.g_bkt + base + s;
        flag = a.g_flag + base;
        pst = a.g_pstart + base;
        psum = a.g_psum + base;
        fcnt = a.g_fcnt + base;
    }
    // ---- bucket sort on |g|^3 in [r2min^1.5, r2max^1.5] ----
    const int nb = n;
    const float lo3 = (float)(a.r2min * sqrt(a.r2min)), hi3 = (float)(a.r2max * sqrt(a.r2max));
    const float scale = (float)nb / (hi3 - lo3);
    for (int i = tid; i <= nb; i += nt) bkt[i] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
        const float qf = d2f_pos(q[i]);
        int b = (int)((qf * sqrtf(qf) - lo3) * scale);
        b = min(max(b, 0), nb - 1);
        atomicAdd(&bkt[b], 1);
    }
    __syncthreads();
    block_excl_scan(bkt, nb, tmp);
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
        const float qf = d2f_pos(q[i]);
        int b = (int)((qf * sqrtf(qf) - lo3) * scale);
        b = min(max(b, 0), nb - 1);
        perm[atomicAdd(&bkt[b], 1)] = i;
    }
    __syncthreads();
    for (int b = tid; b < nb; b += nt) {  // bkt[b] is now the end of bucket b
        const int b0 = b ? bkt[b - 1] : 0, b1 = bkt[b];
        for (int i = b0 + 1; i < b1; i++) {
            const int v = perm[i];
            const double qv = q[v];
            const uint32_t kv = key[v];
            int j = i - 1;
            while (j >= b0 && before(qv, kv, q[perm[j]], key[perm[j]])) {
                perm[j + 1] = perm[j];
                j--;
            }
            perm[j + 1] = v;
        }
    }
    __syncthreads();
    // ---- 2-theta of every reflection in sorted order (Bragg's law) ----
    for (int i = tid; i < n; i += nt) {
        double sth = a.lambda * sqrt(q[perm[i]]) / 2.0;
        if (sth > 1.0) sth = 1.0;
        tt[i] = 2.0 * asin(sth) * (180.0 / kPi);
    }
    __syncthreads();
    // ---- anchor merge ----
    for (int i = tid; i < n; i += nt) flag[i] = (i == 0) || !(tt[i] - tt[i - 1] < a.tol);
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
        if (!flag[i]) continue;
        int anchor = i;
        pst[i] = 1;
        for (int j = i + 1; j < n && !flag[j]; j++) {
            if (!(tt[j] - tt[anchor] < a.tol)) {
                pst[j] = 1;
                anchor = j;
            } else {
                pst[j] = 0;
            }
        }
    }
    __syncthreads();
    // peak starts -> peak ids; bkt becomes the list of peak start positions
    for (int i = tid; i < n; i += nt) fcnt[i] = pst[i];
    __syncthreads();
    const int np = block_excl_scan(pst, n, tmp);
    __syncthreads();
    for (int i = tid; i < n; i += nt)
        if (fcnt[i]) bkt[pst[i]] = i;
    if (tid == 0) bkt[np] = n;
    __syncthreads();
    // ---- per peak: merged intensity (each half-space reflection stands for g and -g) and family count ----
    double lmax = 0.0;
    for (int p = tid; p < np; p += nt) {
        const int i0 = bkt[p], i1 = bkt[p + 1];
        double sum = 0.0;
        int nfam = 0;
        for (int i = i0; i < i1; i++) {
            sum += 2.0 * Ig[perm[i]];
            const uint32_t fk = family_key(key[perm[i]]);
            bool lead = true;
            for (int j = i0; j < i && lead; j++) lead = family_key(key[perm[j]]) != fk;
            nfam += lead;
        }
        psum[p] = sum;
        fcnt[p] = nfam;
        lmax = fmax(lmax, sum);
    }
    const double imax = block_max_double(lmax, dtmp);
    // ---- cutoff, then compaction offsets of kept peaks and their families ----
    for (int p = tid; p < np; p += nt) {
        const bool keep = a.cutoff == 0.0 || psum[p] > a.cutoff * imax;
        flag[p] = keep;
        pst[p] = keep;
        if (!keep) fcnt[p] = 0;
    }
    __syncthreads();
    const int nk = block_excl_scan(pst, np, tmp);
    const int nf = block_excl_scan(fcnt, np, tmp);
    __syncthreads();
    for (int p = tid; p < np; p += nt) {
        if (!flag[p]) continue;
        const int i0 = bkt[p], i1 = bkt[p + 1];
        const int64_t o = base + pst[p];
        a.st_tt[o] = tt[i0];
        a.st_d[o] = 1.0 / sqrt(q[perm[i0]]);
        a.st_I[o] = (a.scaled && imax > 0.0) ? 100.0 * (psum[p] / imax) : psum[p];
        a.st_foff[o] = fcnt[p];
        // families: leaders are first members of each family; rank by descending representative
        for (int i = i0; i < i1; i++) {
            const uint32_t fk = family_key(key[perm[i]]);
            bool lead = true;
            for (int j = i0; j < i && lead; j++) lead = family_key(key[perm[j]]) != fk;
            if (!lead) continue;
            uint32_t rep = 0;
            int cnt = 0;
            for (int j = i0; j < i1; j++)
                if (family_key(key[perm[j]]) == fk) { rep = max(rep, key[perm[j]]); cnt++; }
            int rank = 0;
            for (int m = i0; m < i1; m++) {  // other leaders with a larger representative
                const uint32_t fm = family_key(key[perm[m]]);
                if (fm == fk) continue;
                bool lm = true;
                for (int j = i0; j < m && lm; j++) lm = family_key(key[perm[j]]) != fm;
                if (!lm) continue;
                uint32_t rm = 0;
                for (int j = i0; j < i1; j++)
                    if (family_key(key[perm[j]]) == fm) rm = max(rm, key[perm[j]]);
                rank += rm > rep;
            }
            const int64_t fo = base + fcnt[p] + rank;
            a.st_hkl[3 * fo] = hkl_h(rep);
            a.st_hkl[3 * fo + 1] = hkl_k(rep);
            a.st_hkl[3 * fo + 2] = hkl_l(rep);
            a.st_mult[fo] = 2 * cnt;
        }
    }
    if (tid == 0) {
        a.npk[s] = nk;
        a.nfm[s] = nf;
    }
}

// Exclusive scans of kept peaks and families per structure (single block),
// output capacity check, totals.
__global__ void __launch_bounds__(1024) k_scan_out(const CompactArgs a)
{
    __shared__ long long wp[32], wf[32];
    __shared__ long long cp, cf;
    if (*a.abort_flag) return;
    const int n = a.n_struct;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) { cp = 0; cf = 0; }
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const long long vp = i < n ? a.npk[i] : 0, vf = i < n ? a.nfm[i] : 0;
        long long ip = vp, jf = vf;
        for (int o = 1; o < 32; o <<= 1) {
            const long long x = __shfl_up_sync(0xffffffffu, ip, o), y = __shfl_up_sync(0xffffffffu, jf, o);
            if (lane >= o) { ip += x; jf += y; }
        }
        if (lane == 31) { wp[w] = ip; wf[w] = jf; }
        __syncthreads();
        if (w == 0) {
            const long long x0 = lane < nw ? wp[lane] : 0, y0 = lane < nw ? wf[lane] : 0;
            long long x = x0, y = y0;
            for (int o = 1; o < 32; o <<= 1) {
                const long long u = __shfl_up_sync(0xffffffffu, x, o), v = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) { x += u; y += v; }
            }
            if (lane < nw) { wp[lane] = x - x0; wf[lane] = y - y0; }
        }
        __syncthreads();
        if (i < n) {
            a.out.peak_off[i] = cp + wp[w] + ip - vp;
            a.fam_soff[i] = cf + wf[w] + jf - vf;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) { cp += wp[w] + ip; cf += wf[w] + jf; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.out.peak_off[n] = cp;
        a.fam_soff[n] = cf;
        a.out.totals[1] = cp;
        a.out.totals[2] = cf;
        const int over = cp > a.cap_peaks || cf > a.cap_fam;
        *a.out_abort = over;
        if (over) a.out.totals[3] = n;
        else a.out.fam_off[cp] = cf;
    }
    __syncthreads();
    if (cp > a.cap_peaks || cf > a.cap_fam)
        for (int s = threadIdx.x; s < n; s += blockDim.x) a.out.status[s] = XRD_ECAPACITY;
}

__global__ void __launch_bounds__(128) k_compact(const CompactArgs a)
{
    if (*a.abort_flag || *a.out_abort) return;
    const int s = blockIdx.x;
    const int64_t base = a.refl_off[s], pb = a.out.peak_off[s], fb = a.fam_soff[s];
    const int64_t np = a.npk[s], nf = a.nfm[s];
    for (int64_t p = threadIdx.x; p < np; p += blockDim.x) {
        a.out.two_theta[pb + p] = a.st_tt[base + p];
        a.out.intensity[pb + p] = a.st_I[base + p];
        a.out.d_hkl[pb + p] = a.st_d[base + p];
        a.out.fam_off[pb + p] = fb + a.st_foff[base + p];
    }
    for (int64_t f = threadIdx.x; f < nf; f += blockDim.x) {
        a.out.hkl[3 * (fb + f)] = a.st_hkl[3 * (base + f)];
        a.out.hkl[3 * (fb + f) + 1] = a.st_hkl[3 * (base + f) + 1];
        a.out.hkl[3 * (fb + f) + 2] = a.st_hkl[3 * (base + f) + 2];
        a.out.mult[fb + f] = a.st_mult[base + f];
    }
}

void launch_post(const PostArgs& a, cudaStream_t st)
{
    if (a.n_struct <= 0) return;
    const size_t smem = post_smem_bytes(a.cap_smem);
    cudaFuncSetAttribute(k_post, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_post<<<a.n_struct, kPostThreads, smem, st>>>(a);
}

void launch_compact(const CompactArgs& a, cudaStream_t st)
{
    k_scan_out<<<1, 1024, 0, st>>>(a);
    if (a.n_struct > 0) k_compact<<<a.n_struct, 128, 0, st>>>(a);
}

}  // namespace xrd
