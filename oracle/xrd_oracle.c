/*
 * Plain FP64 CPU oracle for the powder X-ray diffraction pattern.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the CPU
 * baseline leg of the benchmark use it; the product path never does. It
 * shares no code with the CUDA library. Build with -ffp-contract=off so that
 * every product and sum is rounded on its own, as written.
 *
 * Steps follow the list of the method's numerical core in Sec. 2 of the
 * paper; the physics is standard kinematic powder diffraction, which the
 * paper says it does not change (Sec. 1). Each function is the plain
 * definition: no blocking, no reordering, no shortcut (the full sphere of
 * reflections is enumerated, Friedel mates included).
 *
 * Parity pins for each function live in tests/test_oracle_*.py. Agreement with
 * pymatgen's own patterns is parity unpinned: its tabulated scattering-factor
 * coefficients are not available, so every table here is a seeded stand-in
 * passed in by the caller.
 */
#include "xrd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Constant of the atomic scattering-factor expression (Sec. 1, atomic scattering factors). */
#define ORC_F_SCALE 41.78214

/* cos of an angle in degrees. 90, 60 and 120 degrees give their exact cosines. */
static double orc_cosd(double deg)
{
    if (deg == 90.0) return 0.0;
    if (deg == 60.0) return 0.5;
    if (deg == 120.0) return -0.5;
    return cos(deg * (M_PI / 180.0));
}

/*
 * Sec. 2, reciprocal-lattice points: the direct metric tensor
 *   G = [[a^2, ab cos(gamma), ac cos(beta)], [., b^2, bc cos(alpha)], [., ., c^2]]
 * and its inverse, the reciprocal metric Gs, by cofactors over the determinant.
 * |g|^2 = h^T Gs h is the squared length of the reciprocal vector (no 2 pi).
 */
int orc_metric(const double lat[6], double G[6], double Gs[6], double* volume)
{
    const double a = lat[0], b = lat[1], c = lat[2];
    if (!(a > 0.0 && b > 0.0 && c > 0.0) || !isfinite(a) || !isfinite(b) || !isfinite(c)) return -1;
    if (!isfinite(lat[3]) || !isfinite(lat[4]) || !isfinite(lat[5])) return -1;
    const double ca = orc_cosd(lat[3]), cb = orc_cosd(lat[4]), cg = orc_cosd(lat[5]);
    /* volume factor 1 - ca^2 - cb^2 - cg^2 + 2 ca cb cg: the cell is degenerate at 0 */
    const double vf = 1.0 - ca * ca - cb * cb - cg * cg + 2.0 * ca * cb * cg;
    if (!(vf > 1e-6)) return -1;
    const double G11 = a * a, G22 = b * b, G33 = c * c;
    const double G12 = a * b * cg, G13 = a * c * cb, G23 = b * c * ca;
    const double C11 = G22 * G33 - G23 * G23;
    const double C22 = G11 * G33 - G13 * G13;
    const double C33 = G11 * G22 - G12 * G12;
    const double C12 = G13 * G23 - G12 * G33;
    const double C13 = G12 * G23 - G13 * G22;
    const double C23 = G12 * G13 - G11 * G23;
    const double det = G11 * C11 + G12 * C12 + G13 * C13;
    if (G) { G[0] = G11; G[1] = G22; G[2] = G33; G[3] = G12; G[4] = G13; G[5] = G23; }
    Gs[0] = C11 / det; Gs[1] = C22 / det; Gs[2] = C33 / det;
    Gs[3] = C12 / det; Gs[4] = C13 / det; Gs[5] = C23 / det;
    if (volume) *volume = sqrt(det);
    return 0;
}

/* |g|^2 in the method's fixed order: ((G11 hh + G22 kk) + G33 ll) + 2 ((G12 hk + G13 hl) + G23 kl). */
double orc_q(const double Gs[6], int h, int k, int l)
{
    const double hh = (double)(h * h), kk = (double)(k * k), ll = (double)(l * l);
    const double hk = (double)(h * k), hl = (double)(h * l), kl = (double)(k * l);
    const double diag = (Gs[0] * hh + Gs[1] * kk) + Gs[2] * ll;
    const double off = (Gs[3] * hk + Gs[4] * hl) + Gs[5] * kl;
    return diag + 2.0 * off;
}

/* Bragg's law: a reflection at 2-theta has |g| = 2 sin(theta) / lambda. */
double orc_r2(double tt_deg, double lambda)
{
    const double t = 2.0 * sin(tt_deg * (M_PI / 360.0)) / lambda;
    return t * t;
}

static int orc_opts_ok(const orc_opts* o)
{
    return o && o->lambda > 0.0 && isfinite(o->lambda) && o->tt_min >= 0.0 && o->tt_min < o->tt_max &&
           o->tt_max <= 180.0 && o->tt_tol >= 0.0 && o->cutoff >= 0.0 && o->cutoff < 1.0;
}

/*
 * Sec. 2, the reciprocal-lattice points inside the sphere that the 2-theta
 * range reaches: every integer g = (h, k, l) != 0 with
 * r_min^2 <= |g|^2 <= r_max^2. The box |h| <= r_max a (+1) holds the whole
 * sphere because |h| = |g . a| <= |g| a. Loops run h, k, l ascending.
 */
long orc_enumerate(const double lat[6], const orc_opts* o, long cap, int32_t* hkl, double* q)
{
    double Gs[6];
    if (!orc_opts_ok(o) || orc_metric(lat, NULL, Gs, NULL) != 0) return -1;
    const double r2min = orc_r2(o->tt_min, o->lambda), r2max = orc_r2(o->tt_max, o->lambda);
    const double rmax = sqrt(r2max);
    const int H = (int)floor(rmax * lat[0]) + 1, K = (int)floor(rmax * lat[1]) + 1, L = (int)floor(rmax * lat[2]) + 1;
    long n = 0;
    for (int h = -H; h <= H; h++)
        for (int k = -K; k <= K; k++)
            for (int l = -L; l <= L; l++) {
                if (h == 0 && k == 0 && l == 0) continue;
                const double qq = orc_q(Gs, h, k, l);
                if (qq < r2min || qq > r2max) continue;
                if (n < cap) {
                    if (hkl) { hkl[3 * n] = h; hkl[3 * n + 1] = k; hkl[3 * n + 2] = l; }
                    if (q) q[n] = qq;
                }
                n++;
            }
    return n;
}

/*
 * Per-reflection scalars (Sec. 1: Lorentz-polarisation correction):
 *   s = |g| / 2, sin(theta) = lambda |g| / 2 (Bragg), 2-theta in degrees,
 *   LP = (1 + cos^2 2theta) / (sin^2 theta cos theta), d = 1 / |g|.
 */
void orc_refl(double q, double lambda, double* s2, double* tt, double* lp, double* d)
{
    double sth = lambda * sqrt(q) / 2.0;
    if (sth > 1.0) sth = 1.0;
    const double th = asin(sth);
    const double c2 = cos(2.0 * th);
    if (s2) *s2 = q / 4.0;
    if (tt) *tt = 2.0 * th * (180.0 / M_PI);
    if (lp) *lp = (1.0 + c2 * c2) / (sth * sth * cos(th));
    if (d) *d = 1.0 / sqrt(q);
}

/* Atomic scattering factor f(s) = Z - 41.78214 s^2 sum_{i=1..4} a_i exp(-b_i s^2). */
double orc_f(const double* coef, int Z, double s2)
{
    const double* cz = coef + 8 * Z;
    double sum = 0.0;
    for (int i = 0; i < 4; i++) sum += cz[2 * i] * exp(-cz[2 * i + 1] * s2);
    return (double)Z - ORC_F_SCALE * s2 * sum;
}

/*
 * Sec. 2: per reflection, the sum over the atoms' contributions, with the
 * Debye-Waller factor:
 *   F(g) = sum_j occ_j f_j(s) exp(-B_j s^2) [cos 2 pi phi_j + i sin 2 pi phi_j],
 *   phi_j = h x_j + k y_j + l z_j.
 */
void orc_sf(int h, int k, int l, double s2, long n, const double* frac, const int16_t* Z,
            const double* occ, const double* B, const double* coef, double* Fr, double* Fi)
{
    double re = 0.0, im = 0.0;
    for (long j = 0; j < n; j++) {
        const double w = occ[j] * orc_f(coef, Z[j], s2) * exp(-B[j] * s2);
        const double phi = (double)h * frac[3 * j] + (double)k * frac[3 * j + 1] + (double)l * frac[3 * j + 2];
        const double arg = 2.0 * M_PI * phi;
        re += w * cos(arg);
        im += w * sin(arg);
    }
    *Fr = re;
    *Fi = im;
}

typedef struct {
    double q, tt, lp, I, Fr, Fi;
    int h, k, l;
} orc_refl_t;

/* Ascending |g|^2, ties by descending (h, k, l). */
static int orc_cmp(const void* pa, const void* pb)
{
    const orc_refl_t* a = (const orc_refl_t*)pa;
    const orc_refl_t* b = (const orc_refl_t*)pb;
    if (a->q < b->q) return -1;
    if (a->q > b->q) return 1;
    if (a->h != b->h) return a->h > b->h ? -1 : 1;
    if (a->k != b->k) return a->k > b->k ? -1 : 1;
    if (a->l != b->l) return a->l > b->l ? -1 : 1;
    return 0;
}

int orc_is_hexagonal(const double lat[6])
{
    return fabs(lat[3] - 90.0) < 5.0 && fabs(lat[4] - 90.0) < 5.0 && fabs(lat[5] - 120.0) < 5.0 &&
           fabs(lat[0] - lat[1]) < 0.01;
}

/* Family key: the absolute values of the indices sorted in descending order:
 * (h, k, l) padded with 0, or for a hexagonal cell the Miller-Bravais
 * (h, k, i = -h - k, l). */
static void orc_family_key(int h, int k, int l, int hex, int key[4])
{
    int v[4] = {abs(h), abs(k), abs(l), hex ? abs(h + k) : 0};
    for (int i = 0; i < 4; i++)
        for (int j = i + 1; j < 4; j++)
            if (v[j] > v[i]) { int t = v[i]; v[i] = v[j]; v[j] = t; }
    for (int i = 0; i < 4; i++) key[i] = v[i];
}

/* Family key under a caller's point group (the symmetry-aware mode of the
 * calculator-style interface, N3): the family of g is its orbit
 * {M g, -M g : M in the group} (Friedel's law adds the inversion), and its key
 * the lexicographically largest member of the orbit, padded with 0. */
static void orc_family_key_pg(int h, int k, int l, int n_pg, const int32_t* pg, int key[4])
{
    int best[3] = {h, k, l};
    if (-h > best[0] || (-h == best[0] && (-k > best[1] || (-k == best[1] && -l > best[2])))) {
        best[0] = -h; best[1] = -k; best[2] = -l;
    }
    for (int m = 0; m < n_pg; m++) {
        const int32_t* M = pg + 9 * m;
        const int v[3] = {M[0] * h + M[1] * k + M[2] * l, M[3] * h + M[4] * k + M[5] * l,
                          M[6] * h + M[7] * k + M[8] * l};
        for (int sgn = 1; sgn >= -1; sgn -= 2) {
            const int w[3] = {sgn * v[0], sgn * v[1], sgn * v[2]};
            if (w[0] > best[0] || (w[0] == best[0] && (w[1] > best[1] || (w[1] == best[1] && w[2] > best[2])))) {
                best[0] = w[0]; best[1] = w[1]; best[2] = w[2];
            }
        }
    }
    key[0] = best[0]; key[1] = best[1]; key[2] = best[2]; key[3] = 0;
}

/* Lexicographic comparison of signed (h, k, l) triples: >0 when a > b. */
static int orc_lex(const int a[3], const int b[3])
{
    for (int i = 0; i < 3; i++)
        if (a[i] != b[i]) return a[i] > b[i] ? 1 : -1;
    return 0;
}

int orc_pattern(const double lat[6], long n, const double* frac, const int16_t* Z, const double* occ,
                const double* B, const double* coef, int zmax, const orc_opts* o, orc_out* out)
{
    out->n_refl = out->n_peaks_merged = out->n_peaks = out->n_fam = 0;
    out->imax = 0.0;
    if (!orc_opts_ok(o) || n < 0) return 1;
    for (long j = 0; j < n; j++) {
        if (Z[j] < 0 || Z[j] > zmax) return 1;
        if (!isfinite(frac[3 * j]) || !isfinite(frac[3 * j + 1]) || !isfinite(frac[3 * j + 2])) return 1;
        if (!isfinite(occ[j]) || occ[j] < 0.0 || !isfinite(B[j])) return 1;
    }
    double Gs[6];
    if (orc_metric(lat, NULL, Gs, NULL) != 0) return 1;

    /* reflections in the sphere */
    const long nr = orc_enumerate(lat, o, 0, NULL, NULL);
    if (nr < 0) return 1;
    out->n_refl = nr;
    int32_t* hkl = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(nr > 0 ? nr : 1));
    double* qv = (double*)malloc(sizeof(double) * (size_t)(nr > 0 ? nr : 1));
    orc_refl_t* r = (orc_refl_t*)malloc(sizeof(orc_refl_t) * (size_t)(nr > 0 ? nr : 1));
    orc_enumerate(lat, o, nr, hkl, qv);

    /* structure factor, Lorentz-polarisation and intensity of every reflection */
    for (long i = 0; i < nr; i++) {
        double s2, tt, lp;
        orc_refl(qv[i], o->lambda, &s2, &tt, &lp, NULL);
        double Fr, Fi;
        orc_sf(hkl[3 * i], hkl[3 * i + 1], hkl[3 * i + 2], s2, n, frac, Z, occ, B, coef, &Fr, &Fi);
        r[i].q = qv[i]; r[i].tt = tt; r[i].lp = lp; r[i].Fr = Fr; r[i].Fi = Fi;
        r[i].I = (Fr * Fr + Fi * Fi) * lp;
        r[i].h = hkl[3 * i]; r[i].k = hkl[3 * i + 1]; r[i].l = hkl[3 * i + 2];
    }
    free(hkl);
    free(qv);

    /* sort by 2-theta (ascending |g|^2) */
    qsort(r, (size_t)nr, sizeof(orc_refl_t), orc_cmp);
    if (out->cap_refl >= nr) {
        for (long i = 0; i < nr; i++) {
            if (out->refl_hkl) { out->refl_hkl[3 * i] = r[i].h; out->refl_hkl[3 * i + 1] = r[i].k; out->refl_hkl[3 * i + 2] = r[i].l; }
            if (out->refl_q) out->refl_q[i] = r[i].q;
            if (out->refl_tt) out->refl_tt[i] = r[i].tt;
            if (out->refl_lp) out->refl_lp[i] = r[i].lp;
            if (out->refl_I) out->refl_I[i] = r[i].I;
            if (out->refl_Fr) out->refl_Fr[i] = r[i].Fr;
            if (out->refl_Fi) out->refl_Fi[i] = r[i].Fi;
        }
    }

    /*
     * Merge within the angular tolerance: a peak is anchored at the 2-theta of
     * its first reflection; a later reflection joins it while
     * 2theta - anchor < tol, otherwise it opens a new peak.
     */
    long* start = (long*)malloc(sizeof(long) * (size_t)(nr + 1));
    long np = 0;
    for (long i = 0; i < nr; i++) {
        if (np == 0 || !(r[i].tt - r[start[np - 1]].tt < o->tt_tol)) start[np++] = i;
    }
    start[np] = nr;
    out->n_peaks_merged = np;

    double* pI = (double*)malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
    double imax = 0.0;
    for (long p = 0; p < np; p++) {
        double s = 0.0;
        for (long i = start[p]; i < start[p + 1]; i++) s += r[i].I;
        pI[p] = s;
        if (s > imax) imax = s;
    }
    out->imax = imax;

    /* cutoff relative to the largest peak, then scaling to 100 */
    int rc = 0;
    long nk = 0, nf = 0;
    const int hex = orc_is_hexagonal(lat);
    int* fkey = (int*)malloc(sizeof(int) * 4 * (size_t)(nr > 0 ? nr : 1));
    int* frep = (int*)malloc(sizeof(int) * 3 * (size_t)(nr > 0 ? nr : 1));
    int* fmul = (int*)malloc(sizeof(int) * (size_t)(nr > 0 ? nr : 1));
    for (long p = 0; p < np; p++) {
        if (o->cutoff > 0.0 && !(pI[p] > o->cutoff * imax)) continue;
        if (nk >= out->cap_peaks) { rc = 2; break; }
        const long i0 = start[p];
        out->peak_tt[nk] = r[i0].tt;
        out->peak_d[nk] = 1.0 / sqrt(r[i0].q);
        out->peak_I[nk] = (o->scaled && imax > 0.0) ? 100.0 * (pI[p] / imax) : pI[p];
        out->peak_fam_off[nk] = nf;

        /* families: members equal up to permutation and sign of (h, k, l), or of
         * (h, k, i, l) for a hexagonal cell, or in one orbit of the caller's point group */
        long m = 0;
        for (long i = i0; i < start[p + 1]; i++) {
            int key[4], hv[3] = {r[i].h, r[i].k, r[i].l};
            if (o->n_pg > 0) orc_family_key_pg(hv[0], hv[1], hv[2], o->n_pg, o->pg, key);
            else orc_family_key(hv[0], hv[1], hv[2], hex, key);
            long f;
            for (f = 0; f < m; f++)
                if (fkey[4 * f] == key[0] && fkey[4 * f + 1] == key[1] && fkey[4 * f + 2] == key[2] &&
                    fkey[4 * f + 3] == key[3])
                    break;
            if (f == m) {
                for (int t = 0; t < 4; t++) fkey[4 * m + t] = key[t];
                frep[3 * m] = hv[0]; frep[3 * m + 1] = hv[1]; frep[3 * m + 2] = hv[2];
                fmul[m] = 0;
                m++;
            }
            fmul[f] += 1;
            if (orc_lex(hv, &frep[3 * f]) > 0) { frep[3 * f] = hv[0]; frep[3 * f + 1] = hv[1]; frep[3 * f + 2] = hv[2]; }
        }
        /* families of a peak are listed by descending representative */
        for (long a = 0; a < m; a++)
            for (long b = a + 1; b < m; b++)
                if (orc_lex(&frep[3 * b], &frep[3 * a]) > 0) {
                    for (int t = 0; t < 3; t++) { int x = frep[3 * a + t]; frep[3 * a + t] = frep[3 * b + t]; frep[3 * b + t] = x; }
                    int x = fmul[a]; fmul[a] = fmul[b]; fmul[b] = x;
                }
        if (nf + m > out->cap_fam) { rc = 2; break; }
        for (long f = 0; f < m; f++) {
            out->fam_hkl[3 * (nf + f)] = frep[3 * f];
            out->fam_hkl[3 * (nf + f) + 1] = frep[3 * f + 1];
            out->fam_hkl[3 * (nf + f) + 2] = frep[3 * f + 2];
            out->fam_mult[nf + f] = fmul[f];
        }
        nf += m;
        nk++;
    }
    if (rc == 0 && nk <= out->cap_peaks) out->peak_fam_off[nk] = nf;
    out->n_peaks = nk;
    out->n_fam = nf;
    free(fkey); free(frep); free(fmul);
    free(pI); free(start); free(r);
    return rc;
}

/* Gaussian width from the full width at half maximum: FWHM = 2 sqrt(2 ln 2) sigma. */
static double orc_sigma(double fwhm) { return fwhm / (2.0 * sqrt(2.0 * log(2.0))); }

/*
 * Broadened pattern (the differentiable profile used for refinement and for
 * training data with peak broadening, Sec. 1): each reflection of the fixed
 * list adds a unit-height Gaussian of its intensity at its 2-theta.
 */
void orc_broadened(const double lat[6], long n, const double* frac, const int16_t* Z, const double* occ,
                   const double* B, const double* coef, double lambda, long nr, const int32_t* hkl, double t0,
                   double dt, int npts, double fwhm, double* y)
{
    double Gs[6];
    for (int k = 0; k < npts; k++) y[k] = 0.0;
    if (orc_metric(lat, NULL, Gs, NULL) != 0) return;
    const double sg = orc_sigma(fwhm);
    for (long r = 0; r < nr; r++) {
        const int h = hkl[3 * r], k = hkl[3 * r + 1], l = hkl[3 * r + 2];
        double s2, tt, lp, Fr, Fi;
        orc_refl(orc_q(Gs, h, k, l), lambda, &s2, &tt, &lp, NULL);
        orc_sf(h, k, l, s2, n, frac, Z, occ, B, coef, &Fr, &Fi);
        const double I = (Fr * Fr + Fi * Fi) * lp;
        for (int i = 0; i < npts; i++) {
            const double u = t0 + i * dt - tt;
            y[i] += I * exp(-u * u / (2.0 * sg * sg));
        }
    }
}

/* g^T Gs n for integer g and real n (Gs stored as 11, 22, 33, 12, 13, 23). */
static double orc_dot(const double Gs[6], const double g[3], const double n[3])
{
    return g[0] * (Gs[0] * n[0] + Gs[3] * n[1] + Gs[4] * n[2]) + g[1] * (Gs[3] * n[0] + Gs[1] * n[1] + Gs[5] * n[2]) +
           g[2] * (Gs[4] * n[0] + Gs[5] * n[1] + Gs[2] * n[2]);
}

double orc_march_dollase(const double Gs[6], int h, int k, int l, const double po_dir[3], double po_r)
{
    const double g[3] = {(double)h, (double)k, (double)l};
    const double gn = orc_dot(Gs, g, po_dir);
    const double gg = orc_dot(Gs, g, g), nn = orc_dot(Gs, po_dir, po_dir);
    const double c2 = gn * gn / (gg * nn);
    return pow(po_r * po_r * c2 + (1.0 - c2) / po_r, -1.5);
}

void orc_augmented(const double lat[6], long n, const double* frac, const int16_t* Z, const double* occ,
                   const double* B, const double* coef, double lambda, long nr, const int32_t* hkl, double t0,
                   double dt, int npts, double fwhm, double eta, const double po_dir[3], double po_r,
                   const double* z, double sigma, double* y)
{
    double Gs[6];
    for (int k = 0; k < npts; k++) y[k] = 0.0;
    if (orc_metric(lat, NULL, Gs, NULL) != 0) return;
    const double cl = eta * 2.0 / (M_PI * fwhm);
    const double cg = (1.0 - eta) * (2.0 / fwhm) * sqrt(log(2.0) / M_PI);
    for (long r = 0; r < nr; r++) {
        const int h = hkl[3 * r], k = hkl[3 * r + 1], l = hkl[3 * r + 2];
        double s2, tt, lp, Fr, Fi;
        orc_refl(orc_q(Gs, h, k, l), lambda, &s2, &tt, &lp, NULL);
        orc_sf(h, k, l, s2, n, frac, Z, occ, B, coef, &Fr, &Fi);
        const double I = (Fr * Fr + Fi * Fi) * lp * orc_march_dollase(Gs, h, k, l, po_dir, po_r);
        for (int i = 0; i < npts; i++) {
            const double u = t0 + i * dt - tt;
            const double x2 = 4.0 * u * u / (fwhm * fwhm);
            y[i] += I * (cl / (1.0 + x2) + cg * exp(-log(2.0) * x2));
        }
    }
    if (z)
        for (int i = 0; i < npts; i++) y[i] += sigma * sqrt(y[i] > 0.0 ? y[i] : 0.0) * z[i];
}

/* d f(s) / d s^2 = -41.78214 sum_i a_i exp(-b_i s^2) (1 - b_i s^2). */
static double orc_fprime(const double* coef, int Z, double s2)
{
    const double* cz = coef + 8 * Z;
    double sum = 0.0;
    for (int i = 0; i < 4; i++) sum += cz[2 * i] * exp(-cz[2 * i + 1] * s2) * (1.0 - cz[2 * i + 1] * s2);
    return -ORC_F_SCALE * sum;
}

/* Derivative of the direct metric G with respect to lattice parameter m
 * (0..2: a, b, c in angstrom; 3..5: alpha, beta, gamma in degrees), as a full 3x3. */
static void orc_dG(const double lat[6], int m, double D[3][3])
{
    const double a = lat[0], b = lat[1], c = lat[2];
    const double ca = orc_cosd(lat[3]), cb = orc_cosd(lat[4]), cg = orc_cosd(lat[5]);
    const double rad = M_PI / 180.0;
    memset(D, 0, sizeof(double) * 9);
    switch (m) {
    case 0: D[0][0] = 2 * a; D[0][1] = D[1][0] = b * cg; D[0][2] = D[2][0] = c * cb; break;
    case 1: D[1][1] = 2 * b; D[0][1] = D[1][0] = a * cg; D[1][2] = D[2][1] = c * ca; break;
    case 2: D[2][2] = 2 * c; D[0][2] = D[2][0] = a * cb; D[1][2] = D[2][1] = b * ca; break;
    case 3: D[1][2] = D[2][1] = -b * c * sin(lat[3] * rad) * rad; break;
    case 4: D[0][2] = D[2][0] = -a * c * sin(lat[4] * rad) * rad; break;
    default: D[0][1] = D[1][0] = -a * b * sin(lat[5] * rad) * rad; break;
    }
}

void orc_broadened_grad(const double lat[6], long n, const double* frac, const int16_t* Z, const double* occ,
                        const double* B, const double* coef, double lambda, long nr, const int32_t* hkl, double t0,
                        double dt, int npts, double fwhm, const double* dLdy, double* dfrac, double* dB,
                        double* dlat)
{
    double Gs[6];
    for (long j = 0; j < 3 * n; j++) dfrac[j] = 0.0;
    for (long j = 0; j < n; j++) dB[j] = 0.0;
    for (int m = 0; m < 6; m++) dlat[m] = 0.0;
    if (orc_metric(lat, NULL, Gs, NULL) != 0) return;
    const double S[3][3] = {{Gs[0], Gs[3], Gs[4]}, {Gs[3], Gs[1], Gs[5]}, {Gs[4], Gs[5], Gs[2]}};
    double dG[6][3][3];
    for (int m = 0; m < 6; m++) orc_dG(lat, m, dG[m]);
    const double sg = orc_sigma(fwhm);
    const double l2 = lambda * lambda / 4.0;
    for (long r = 0; r < nr; r++) {
        const int hv[3] = {hkl[3 * r], hkl[3 * r + 1], hkl[3 * r + 2]};
        const double q = orc_q(Gs, hv[0], hv[1], hv[2]);
        double s2, tt, lp, Fr, Fi;
        orc_refl(q, lambda, &s2, &tt, &lp, NULL);
        orc_sf(hv[0], hv[1], hv[2], s2, n, frac, Z, occ, B, coef, &Fr, &Fi);
        const double I = (Fr * Fr + Fi * Fi) * lp;
        /* dL/dI and dL/d(2theta) from the Gaussians */
        double dLdI = 0.0, dLdT = 0.0;
        for (int i = 0; i < npts; i++) {
            const double u = t0 + i * dt - tt;
            const double g = exp(-u * u / (2.0 * sg * sg));
            dLdI += dLdy[i] * g;
            dLdT += dLdy[i] * I * g * u / (sg * sg);
        }
        /* atoms: dF/dx_j = 2 pi i h w_j e^{i phi_j}, dF/dB_j = -s^2 w_j e^{i phi_j}; dI = 2 lp Re(conj(F) dF) */
        double dFq_r = 0.0, dFq_i = 0.0; /* dF/dq */
        for (long j = 0; j < n; j++) {
            const double f = orc_f(coef, Z[j], s2), dw = exp(-B[j] * s2);
            const double w = occ[j] * f * dw;
            const double phi = 2.0 * M_PI * ((double)hv[0] * frac[3 * j] + (double)hv[1] * frac[3 * j + 1] +
                                             (double)hv[2] * frac[3 * j + 2]);
            const double c = cos(phi), s = sin(phi);
            /* Re(conj(F) * i * w e^{i phi}) = w (Fi c - Fr s) */
            const double im_part = w * (Fi * c - Fr * s);
            for (int d = 0; d < 3; d++) dfrac[3 * j + d] += dLdI * 2.0 * lp * 2.0 * M_PI * hv[d] * im_part;
            dB[j] += dLdI * 2.0 * lp * (-s2) * w * (Fr * c + Fi * s);
            const double dwds2 = occ[j] * dw * (orc_fprime(coef, Z[j], s2) - B[j] * f);
            dFq_r += 0.25 * dwds2 * c;
            dFq_i += 0.25 * dwds2 * s;
        }
        /* lattice: through |g|^2 into s^2 (f, Debye-Waller), LP and 2-theta */
        const double X = l2 * q;
        const double c2 = 1.0 - 2.0 * X, rt = sqrt(1.0 - X);
        const double N = 1.0 + c2 * c2, D = X * rt;
        const double dN = -4.0 * c2, dD = rt - X / (2.0 * rt);
        const double dlp_dq = (dN * D - N * dD) / (D * D) * l2;
        const double dT_dq = (360.0 / M_PI) / (2.0 * sqrt(X) * rt) * l2;
        const double dI_dq = 2.0 * lp * (Fr * dFq_r + Fi * dFq_i) + (Fr * Fr + Fi * Fi) * dlp_dq;
        const double dLdq = dLdI * dI_dq + dLdT * dT_dq;
        /* dq/dp = -v^T (dG/dp) v with v = G* h */
        double v[3];
        for (int a = 0; a < 3; a++) v[a] = S[a][0] * hv[0] + S[a][1] * hv[1] + S[a][2] * hv[2];
        for (int m = 0; m < 6; m++) {
            double qf = 0.0;
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) qf += v[a] * dG[m][a][b] * v[b];
            dlat[m] += dLdq * (-qf);
        }
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_pattern_batch(int n_struct, const double* lattice, const int64_t* atom_off, const double* frac,
                      const int16_t* Z, const double* occ, const double* B, const double* coef, int zmax,
                      const orc_opts* o, int threads, int count_only, int64_t* refl_count,
                      const int64_t* cap_off, double* peak_tt, double* peak_I, double* peak_d,
                      int64_t* peak_fam_off, int32_t* fam_hkl, int32_t* fam_mult,
                      int64_t* n_peaks, int64_t* n_fam, int32_t* status)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int s = 0; s < n_struct; s++) {
        if (count_only) {
            const long c = orc_enumerate(lattice + 6 * s, o, 0, NULL, NULL);
            refl_count[s] = c < 0 ? 0 : c;
            if (status) status[s] = c < 0 ? 1 : 0;
            bad |= c < 0;
            continue;
        }
        const long a0 = (long)atom_off[s], na = (long)(atom_off[s + 1] - atom_off[s]);
        const long base = (long)cap_off[s];
        const long cap = (long)refl_count[s];
        /* per-peak family offsets are relative to the structure's family slice;
         * peak p's families end at the next peak's offset, the last at n_fam[s] */
        int64_t* tmp_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cap + 1));
        orc_out out;
        memset(&out, 0, sizeof(out));
        out.cap_peaks = cap; out.cap_fam = cap;
        out.peak_tt = peak_tt + base; out.peak_I = peak_I + base; out.peak_d = peak_d + base;
        out.peak_fam_off = tmp_off;
        out.fam_hkl = fam_hkl + 3 * base; out.fam_mult = fam_mult + base;
        const int rc = orc_pattern(lattice + 6 * s, na, frac + 3 * a0, Z + a0, occ + a0, B + a0, coef, zmax, o, &out);
        for (long p = 0; p < out.n_peaks; p++) peak_fam_off[base + p] = tmp_off[p];
        free(tmp_off);
        n_peaks[s] = out.n_peaks;
        n_fam[s] = out.n_fam;
        if (status) status[s] = rc;
        bad |= rc != 0;
    }
    return bad;
}
