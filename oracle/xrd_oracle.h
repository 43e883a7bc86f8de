/*
 * Plain FP64 CPU oracle for the powder X-ray diffraction pattern.
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the package smoke check and the CPU
 * baseline leg of the benchmark call this code; the CUDA product path never
 * does, and the two share no source, header, table or helper.
 *
 * Every function computes the plain definition, step by step, in double
 * precision with libm, in the order the paper lists the steps (Sec. 2):
 * reciprocal-lattice points inside the sphere, the structure-factor sum over
 * atoms, the Lorentz-polarisation and Debye-Waller factors, merging of
 * reflections within the angular tolerance, grouping of equivalent
 * reflections into hkl families, then the optional intensity cutoff of
 * Sec. 2 and the 0-100 scaling of Sec. 3.
 *
 * Layouts: lattice = (a, b, c, alpha, beta, gamma), lengths in angstrom,
 * angles in degrees; metric tensors are stored as (11, 22, 33, 12, 13, 23);
 * coef = [zmax + 1][4][2] holding (a_i, b_i) of each element.
 */
#ifndef XRD_ORACLE_H
#define XRD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double lambda;   /* wavelength, angstrom */
    double tt_min;   /* 2-theta range, degrees, inclusive */
    double tt_max;
    double tt_tol;   /* merge tolerance, degrees */
    double cutoff;   /* keep peaks with I > cutoff * Imax; 0 keeps all */
    int scaled;      /* 1: scale intensities so that the largest is 100 */
    int n_pg;        /* 0: families by permutation and sign (R5, R17); > 0: by the point group below */
    const int32_t* pg; /* [n_pg][3][3] integer operations on (h, k, l) as a column vector */
} orc_opts;

/* Direct metric G and reciprocal metric Gs = G^-1; returns 0, or -1 for an invalid cell. */
int orc_metric(const double lat[6], double G[6], double Gs[6], double* volume);

/* |g|^2 = h^T Gs h in the fixed evaluation order of the method. */
double orc_q(const double Gs[6], int h, int k, int l);

/* (2 sin(theta)/lambda)^2 for a 2-theta value in degrees. */
double orc_r2(double tt_deg, double lambda);

/* Full-sphere enumeration by a plain box loop; writes up to cap entries, returns the count. */
long orc_enumerate(const double lat[6], const orc_opts* o, long cap, int32_t* hkl, double* q);

/* Per-reflection scalars from |g|^2: s^2, 2-theta (deg), Lorentz-polarisation factor, d. */
void orc_refl(double q, double lambda, double* s2, double* tt, double* lp, double* d);

/* Atomic scattering factor f(s) of element Z from its (a_i, b_i) table. */
double orc_f(const double* coef, int Z, double s2);

/* Structure factor F(g) = sum_j occ_j f_j(s) exp(-B_j s^2) exp(2 pi i g.x_j). */
void orc_sf(int h, int k, int l, double s2, long n, const double* frac, const int16_t* Z,
            const double* occ, const double* B, const double* coef, double* Fr, double* Fi);

typedef struct {
    /* capacities (inputs) */
    long cap_refl, cap_peaks, cap_fam;
    /* full-sphere reflections sorted by (q, -h, -k, -l); any pointer may be NULL */
    int32_t* refl_hkl; double* refl_q; double* refl_tt; double* refl_lp; double* refl_I;
    double* refl_Fr; double* refl_Fi;
    /* peaks after cutoff and scaling, ascending 2-theta */
    double* peak_tt; double* peak_I; double* peak_d; int64_t* peak_fam_off; /* [cap_peaks + 1] */
    /* hkl families: representative (h, k, l) and multiplicity */
    int32_t* fam_hkl; int32_t* fam_mult;
    /* counts (outputs) */
    long n_refl, n_peaks_merged, n_peaks, n_fam;
    double imax; /* largest merged-peak intensity before scaling */
} orc_out;

/* One structure, every step; returns 0, 1 (invalid input) or 2 (capacity too small). */
int orc_pattern(const double lat[6], long n, const double* frac, const int16_t* Z, const double* occ,
                const double* B, const double* coef, int zmax, const orc_opts* o, orc_out* out);

/* Batch of structures, OpenMP across structures when threads > 1.
 * refl_count[s] is the full-sphere reflection count (output); the per-structure
 * output capacity for peaks and families is cap[s] = refl_count[s] and the
 * per-structure slices start at cap_off[s] (exclusive prefix sum of cap). Pass
 * count_only = 1 to fill refl_count only. status[s] gets orc_pattern's code. */
int orc_pattern_batch(int n_struct, const double* lattice, const int64_t* atom_off, const double* frac,
                      const int16_t* Z, const double* occ, const double* B, const double* coef, int zmax,
                      const orc_opts* o, int threads, int count_only, int64_t* refl_count,
                      const int64_t* cap_off, double* peak_tt, double* peak_I, double* peak_d,
                      int64_t* peak_fam_off, int32_t* fam_hkl, int32_t* fam_mult,
                      int64_t* n_peaks, int64_t* n_fam, int32_t* status);

/*
 * Gaussian-broadened pattern of one structure over a fixed list of full-sphere
 * reflections hkl[nr][3] (no merge, no cutoff, no scaling):
 *   y_k = sum_r I_r exp(-(t_k - 2theta_r)^2 / (2 sigma^2)),  t_k = t0 + k dt,
 *   sigma = fwhm / (2 sqrt(2 ln 2)).
 * Every grid point sees every reflection (no window).
 */
void orc_broadened(const double lat[6], long n, const double* frac, const int16_t* Z, const double* occ,
                   const double* B, const double* coef, double lambda, long nr, const int32_t* hkl, double t0,
                   double dt, int npts, double fwhm, double* y);

/* Analytic gradient of L = sum_k dLdy_k y_k (same fixed list) with respect to the
 * fractional coordinates dfrac[n][3], the B factors dB[n] and the lattice
 * parameters dlat[6] (per angstrom and per degree). Outputs are overwritten. */
void orc_broadened_grad(const double lat[6], long n, const double* frac, const int16_t* Z, const double* occ,
                        const double* B, const double* coef, double lambda, long nr, const int32_t* hkl, double t0,
                        double dt, int npts, double fwhm, const double* dLdy, double* dfrac, double* dB,
                        double* dlat);

/*
 * Augmented pattern (Sec. 1: training sets for ML models are patterns modified
 * with broadening, noise and preferred orientation; the paper gives no formulas,
 * so these are the standard textbook forms): every reflection of the
 * fixed list adds its intensity I = |F|^2 LP, times the March-Dollase factor
 *   P = (r^2 cos^2(alpha) + sin^2(alpha) / r)^(-3/2),
 * alpha the angle between g and the reciprocal-lattice direction po_dir (g.n and
 * |g|, |n| in the reciprocal metric), times an area-normalised pseudo-Voigt of
 * full width at half maximum fwhm (degrees) and Lorentzian fraction eta,
 *   PV(u) = eta (2 / (pi fwhm)) / (1 + 4 u^2 / fwhm^2)
 *         + (1 - eta) (2 / fwhm) sqrt(ln 2 / pi) exp(-4 ln 2 u^2 / fwhm^2),
 * u = t - 2theta, at every grid point (no window). Then, when z is not NULL,
 * y_k += sigma sqrt(max(y_k, 0)) z_k (z: the caller's standard normal draws).
 */
void orc_augmented(const double lat[6], long n, const double* frac, const int16_t* Z, const double* occ,
                   const double* B, const double* coef, double lambda, long nr, const int32_t* hkl, double t0,
                   double dt, int npts, double fwhm, double eta, const double po_dir[3], double po_r,
                   const double* z, double sigma, double* y);

/* March-Dollase factor of one reflection (h, k, l) about po_dir in reciprocal metric Gs. */
double orc_march_dollase(const double Gs[6], int h, int k, int l, const double po_dir[3], double po_r);

/*
 * 1 when the cell is hexagonal in the standard setting: alpha and beta within
 * 5 degrees of 90, gamma within 5 degrees of 120, |a - b| < 0.01 angstrom.
 * Families of such a cell group reflections by permutation and sign of the
 * Miller-Bravais indices (h, k, i = -h - k, l) (the 4-index convention of the
 * pymatgen calculator the paper accelerates, Sec. 2), else of (h, k, l).
 */
int orc_is_hexagonal(const double lat[6]);

/* Number of threads OpenMP would use for threads = 0 (all cores). */
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
