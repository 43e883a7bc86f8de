// Steps S7-S8: Gaussian-broadened pattern and its adjoint.
//
// The broadened profile y_k = sum_g I_g exp(-(t_k - 2theta_g)^2 / (2 sigma^2))
// is the differentiable form of the pattern used for refinement and for
// training patterns with peak broadening (Sec. 1). Each Friedel-unique
// reflection stands for g and -g (weight 2). Every Gaussian is cut to the grid
// points b - W .. b + W + 1 around its grid cell b, W = ceil(6 sigma / dt), in
// the forward and the backward pass alike, so the gradient is the exact
// gradient of the computed y.
//
// Adjoint, per reflection r (F, dF/ds^2 saved by the forward pass):
//   dL/dI_r = 2 sum_k g_k G_rk,  dL/d2theta_r = 2 I_r sum_k g_k G_rk (t_k - 2theta_r) / sigma^2,
//   dI/dx_j = 4 pi h LP w_j (Im F cos phi_j - Re F sin phi_j)   (likewise y with k, z with l),
//   dI/dB_j = -2 LP s^2 w_j (Re F cos phi_j + Im F sin phi_j),
//   dI/dq  = LP Re(conj F dF/ds^2) / 2 + |F|^2 dLP/dq,  q = |g|^2 = h^T G* h,
//   dL/dG* = sum_r dL/dq_r h h^T,  dL/dG = -G* (dL/dG*) G*,  then G(a, b, c, alpha, beta, gamma).
#include <cmath>

#include "xrd_internal.cuh"
#include "xrd_launch.h"

namespace xrd {

constexpr int kGradThreads = 256;
constexpr int kAtomChunkRefl = 1024;  // reflections staged per chunk in k_grad_atoms
constexpr float kLog2e = 1.4426950408889634f;

// ---------------------------------------------------------------- forward: broadened pattern

__global__ void __launch_bounds__(kGradThreads) k_broaden(const GradArgs a)
{
    pdl_enter();
    extern __shared__ int bins[];  // cell counts, then offsets; cells c = b + W + 1 in [0, nb)
    __shared__ int tmp[34];
    const int s = blockIdx.x;
    float* __restrict__ yo = a.y + (int64_t)s * a.n_pts;
    if (*a.abort_flag) {
        for (int k = threadIdx.x; k < a.n_pts; k += blockDim.x) yo[k] = 0.f;
        return;
    }
    const int64_t base = a.refl_off[s];
    const int n = (int)(a.refl_off[s + 1] - base);
    const int W = a.W, nb = a.n_pts + 2 * W + 2;
    const float cg = (float)(kLog2e / (2.0 * a.sigma * a.sigma));
    // cell and fractional offset of every reflection's 2theta on the grid
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double T = two_theta_q(a.q[base + i], a.l2h, a.l2l, a.ttab);
        const double pos = (T - a.t0) / a.dt;
        const double fb = floor(pos);
        int b;
        float d;
        if (fb < (double)(-W - 1) || fb > (double)(a.n_pts + W)) {
            b = INT_MIN;  // no grid point within the window
            d = 0.f;
        } else {
            b = (int)fb;
            d = (float)(pos - fb);
        }
        a.tb[base + i] = b;
        a.td[base + i] = d;
    }
    for (int c = threadIdx.x; c <= nb; c += blockDim.x) bins[c] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int b = a.tb[base + i];
        if (b != INT_MIN) atomicAdd(&bins[b + W + 1], 1);
    }
    __syncthreads();
    block_excl_scan(bins, nb, tmp);
    __syncthreads();
    int* __restrict__ perm = a.perm + base;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int b = a.tb[base + i];
        if (b != INT_MIN) perm[atomicAdd(&bins[b + W + 1], 1)] = i;
    }
    __syncthreads();
    // bins[c] is now the end of cell c; order each cell by reflection index (deterministic sums)
    for (int c = threadIdx.x; c < nb; c += blockDim.x) {
        const int c0 = c ? bins[c - 1] : 0, c1 = bins[c];
        for (int i = c0 + 1; i < c1; i++) {
            const int v = perm[i];
            int j = i - 1;
            while (j >= c0 && perm[j] > v) {
                perm[j + 1] = perm[j];
                j--;
            }
            perm[j + 1] = v;
        }
    }
    __syncthreads();
    // gather: grid point k sees the reflections of cells b in [k - W - 1, k + W]
    const float dt = (float)a.dt;
    for (int k = threadIdx.x; k < a.n_pts; k += blockDim.x) {
        float acc = 0.f;
        const int c_lo = k, c_hi = k + 2 * W + 1;  // cells c = b + W + 1
        const int i0 = c_lo ? bins[c_lo - 1] : 0, i1 = bins[c_hi];
        for (int i = i0; i < i1; i++) {
            const int r = perm[i];
            const float u = ((float)(k - a.tb[base + r]) - a.td[base + r]) * dt;
            acc = fmaf(2.f * a.Ig[base + r], ex2_approx(-u * u * cg), acc);
        }
        yo[k] = acc;
    }
}

// ---------------------------------------------------------------- backward: per reflection + lattice

__device__ __forceinline__ void dG_dp(const double* lat, int m, double D[3][3])
{
    const double a = lat[0], b = lat[1], c = lat[2];
    const double rad = kPi / 180.0;
    const double ca = cos(lat[3] * rad), cb = cos(lat[4] * rad), cg = cos(lat[5] * rad);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) D[i][j] = 0.0;
    switch (m) {
    case 0: D[0][0] = 2 * a; D[0][1] = D[1][0] = b * cg; D[0][2] = D[2][0] = c * cb; break;
    case 1: D[1][1] = 2 * b; D[0][1] = D[1][0] = a * cg; D[1][2] = D[2][1] = c * ca; break;
    case 2: D[2][2] = 2 * c; D[0][2] = D[2][0] = a * cb; D[1][2] = D[2][1] = b * ca; break;
    case 3: D[1][2] = D[2][1] = -b * c * sin(lat[3] * rad) * rad; break;
    case 4: D[0][2] = D[2][0] = -a * c * sin(lat[4] * rad) * rad; break;
    default: D[0][1] = D[1][0] = -a * b * sin(lat[5] * rad) * rad; break;
    }
}

__global__ void __launch_bounds__(kGradThreads) k_grad_refl(const GradArgs a)
{
    pdl_enter();
    __shared__ double red[6][kGradThreads / 32];
    const int s = blockIdx.x;
    const bool ok = !*a.abort_flag && a.geo[s].status == XRD_OK;
    const int64_t base = a.refl_off[s];
    const int n = ok ? (int)(a.refl_off[s + 1] - base) : 0;
    const int W = a.W;
    const float cg = (float)(kLog2e / (2.0 * a.sigma * a.sigma));
    const float inv_s2 = (float)(1.0 / (a.sigma * a.sigma));
    const float dt = (float)a.dt, l2 = (float)a.l2d;
    const float* __restrict__ g = a.dLdy + (int64_t)s * a.n_pts;
    double m6[6] = {0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t r = base + i;
        const int b = a.tb[r];
        float sI = 0.f, sT = 0.f;
        if (b != INT_MIN) {
            const float d = a.td[r];
            const int k0 = max(0, b - W), k1 = min(a.n_pts - 1, b + W + 1);
            for (int k = k0; k <= k1; k++) {
                const float u = ((float)(k - b) - d) * dt;
                const float G = ex2_approx(-u * u * cg);
                sI = fmaf(g[k], G, sI);
                sT = fmaf(g[k] * G, u, sT);
            }
        }
        const float4 F = a.Fx[r];
        const float I = a.Ig[r];
        const float dLdI = 2.f * sI;
        const float dLdT = 2.f * I * sT * inv_s2;
        const double qd = a.q[r];
        const float qf = d2f_pos(qd);
        const float X = qf * l2;  // sin^2 theta
        float cc = 1.f - X;       // cos^2 theta; above 2theta = 90 degrees from |g|^2 in FP64 (cancellation)
        if (X > 0.5f) cc = fmaxf((float)fma(-a.l2d, qd, 1.0), (float)kCos90Sq);
        const float c2 = fmaf(-2.f, X, 1.f), rt = sqrtf(cc);
        const float N = fmaf(c2, c2, 1.f), D = X * rt;
        const float lp = N / D;
        const float dlp = (-4.f * c2 * D - N * (rt - X / (2.f * rt))) / (D * D) * l2;
        const float dT = (float)(360.0 / kPi) / (2.f * sqrtf(X) * rt) * l2;
        const float alpha = dLdI * lp;
        a.U[r] = alpha * F.x;
        a.V[r] = alpha * F.y;
        const float FF = fmaf(F.x, F.x, F.y * F.y);
        const float dIdq = fmaf(0.5f * lp, fmaf(F.x, F.z, F.y * F.w), FF * dlp);
        const double wq = f2d_fast(fmaf(dLdI, dIdq, dLdT * dT));
        const uint32_t key = a.key[r];
        const double h = i2d_exact(hkl_h(key)), k = i2d_exact(hkl_k(key)), l = i2d_exact(hkl_l(key));
        m6[0] += wq * h * h;
        m6[1] += wq * k * k;
        m6[2] += wq * l * l;
        m6[3] += wq * h * k;
        m6[4] += wq * h * l;
        m6[5] += wq * k * l;
    }
    // deterministic block reduction of the six sums
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = 0; c < 6; c++) {
        double v = m6[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[c][w] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    float* __restrict__ out = a.d_lat + 6 * (int64_t)s;
    if (!ok) {
        for (int c = 0; c < 6; c++) out[c] = 0.f;
        return;
    }
    double M6[6];
    for (int c = 0; c < 6; c++) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += red[c][i];
        M6[c] = t;
    }
    // dL/dG* as a full symmetric matrix (q = sum over all a, b of G*_ab h_a h_b)
    const double M[3][3] = {{M6[0], M6[3], M6[4]}, {M6[3], M6[1], M6[5]}, {M6[4], M6[5], M6[2]}};
    const double* gs = a.geo[s].gs;
    const double S[3][3] = {{gs[0], gs[3], gs[4]}, {gs[3], gs[1], gs[5]}, {gs[4], gs[5], gs[2]}};
    double SM[3][3], DG[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double t = 0.0;
            for (int m = 0; m < 3; m++) t += S[i][m] * M[m][j];
            SM[i][j] = t;
        }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double t = 0.0;
            for (int m = 0; m < 3; m++) t += SM[i][m] * S[m][j];
            DG[i][j] = -t;  // dL/dG = -G* (dL/dG*) G*
        }
    const double* lat = a.lattice + 6 * (int64_t)s;
    for (int p = 0; p < 6; p++) {
        double D[3][3];
        dG_dp(lat, p, D);
        double t = 0.0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) t += DG[i][j] * D[i][j];
        out[p] = (float)t;
    }
}

// ---------------------------------------------------------------- backward: atoms

// One CTA per structure. Thread t owns atom t mod Nc of the current atom chunk
// and every P-th reflection (residue t / Nc); partial sums are reduced over the
// residues in a fixed order.
__global__ void __launch_bounds__(kGradThreads) k_grad_atoms(const GradArgs a)
{
    pdl_enter();
    __shared__ uint32_t skey[kAtomChunkRefl];
    __shared__ float ss2[kAtomChunkRefl], sU[kAtomChunkRefl], sV[kAtomChunkRefl];
    __shared__ float red[kGradThreads][4];
    const int s = blockIdx.x;
    const int64_t j0 = a.atom_off[s], j1 = a.atom_off[s + 1];
    const int N = (int)(j1 - j0);
    const bool ok = !*a.abort_flag && a.geo[s].status == XRD_OK;
    if (!ok) {
        if (j0 < 0 || j1 > a.n_atoms || N < 0) return;  // invalid atom offsets: touch nothing
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            a.d_frac[3 * (j0 + i)] = a.d_frac[3 * (j0 + i) + 1] = a.d_frac[3 * (j0 + i) + 2] = 0.f;
            a.d_B[j0 + i] = 0.f;
        }
        return;
    }
    const int64_t rb = a.refl_off[s];
    const int nr = (int)(a.refl_off[s + 1] - rb);
    const int Nc = min(N, (int)blockDim.x);
    if (Nc == 0) return;
    const int P = blockDim.x / Nc;
    const int t = threadIdx.x;
    const int rho = t / Nc;
    for (int ac0 = 0; ac0 < N; ac0 += Nc) {
        const int al = t % Nc;
        const int at_i = ac0 + al;
        const bool valid = rho < P && at_i < N;
        Atom32 at{};
        Coef32 c{};
        if (valid) {
            at = a.atom32[j0 + at_i];
            c = a.coef32[at.z];
        }
        float gx = 0.f, gy = 0.f, gz = 0.f, gB = 0.f;
        for (int r0 = 0; r0 < nr; r0 += kAtomChunkRefl) {
            const int nc = min(kAtomChunkRefl, nr - r0);
            __syncthreads();
            for (int i = t; i < nc; i += blockDim.x) {
                skey[i] = a.key[rb + r0 + i];
                ss2[i] = d2f_pos(a.q[rb + r0 + i]) * 0.25f;
                sU[i] = a.U[rb + r0 + i];
                sV[i] = a.V[rb + r0 + i];
            }
            __syncthreads();
            if (valid) {
                for (int i = rho; i < nc; i += P) {
                    const uint32_t key = skey[i];
                    const int h = hkl_h(key), k = hkl_k(key), l = hkl_l(key);
                    const uint32_t Ph = (uint32_t)h * at.X + (uint32_t)k * at.Y + (uint32_t)l * at.Z;
                    float sn, cs;
                    __sincosf((float)(int32_t)Ph * 1.4629180792671596e-09f, &sn, &cs);
                    const float s2 = ss2[i];
                    const float e0 = ex2_approx(c.bl[0] * s2), e1 = ex2_approx(c.bl[1] * s2);
                    const float e2 = ex2_approx(c.bl[2] * s2), e3 = ex2_approx(c.bl[3] * s2);
                    const float f = fmaf(s2, fmaf(c.a[0], e0, fmaf(c.a[1], e1, fmaf(c.a[2], e2, c.a[3] * e3))),
                                         (float)at.z);
                    const float w = f * ex2_approx(fmaf(at.nb, s2, at.lo));
                    const float U = sU[i], V = sV[i];
                    const float t1 = w * fmaf(V, cs, -U * sn);
                    const float t2 = w * fmaf(U, cs, V * sn);
                    gx = fmaf((float)h, t1, gx);
                    gy = fmaf((float)k, t1, gy);
                    gz = fmaf((float)l, t1, gz);
                    gB = fmaf(s2, t2, gB);
                }
            }
        }
        red[t][0] = gx;
        red[t][1] = gy;
        red[t][2] = gz;
        red[t][3] = gB;
        __syncthreads();
        if (rho == 0 && at_i < N) {
            float sx = 0.f, sy = 0.f, sz = 0.f, sb = 0.f;
            for (int p = 0; p < P; p++) {
                const float* v = red[p * Nc + al];
                sx += v[0];
                sy += v[1];
                sz += v[2];
                sb += v[3];
            }
            const int64_t o = j0 + at.src;
            const float fourpi = (float)(4.0 * kPi);
            a.d_frac[3 * o] = fourpi * sx;
            a.d_frac[3 * o + 1] = fourpi * sy;
            a.d_frac[3 * o + 2] = fourpi * sz;
            a.d_B[o] = -2.f * sb;
        }
        __syncthreads();
    }
}

size_t broaden_smem_bytes(int n_pts, int W) { return sizeof(int) * (size_t)(n_pts + 2 * W + 3); }

void launch_broaden(const GradArgs& a, cudaStream_t st)
{
    if (a.n_struct <= 0) return;
    const size_t smem = broaden_smem_bytes(a.n_pts, a.W);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_broaden, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    launch_pdl(k_broaden, a.n_struct, kGradThreads, smem, st, a);
}

void launch_grad(const GradArgs& a, cudaStream_t st)
{
    if (a.n_struct <= 0) return;
    k_grad_refl<<<a.n_struct, kGradThreads, 0, st>>>(a);
    launch_pdl(k_grad_atoms, a.n_struct, kGradThreads, 0, st, a);
}

}  // namespace xrd
