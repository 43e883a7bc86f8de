/*
 * xrd.h -- C ABI of the GB300 powder X-ray diffraction pattern engine.
 *
 * The library computes, for a batch of crystal structures, the powder
 * diffraction pattern of each one: the steps of the numerical core listed in
 * Sec. 2 of arXiv 2602.11709 (reciprocal-lattice points inside the accessible
 * sphere, structure-factor sums over atoms, Lorentz-polarisation and
 * Debye-Waller factors, merging of reflections within an angular tolerance,
 * grouping of equivalent reflections into hkl families), followed by the
 * optional intensity cutoff (Sec. 2) and the 0-100 scaling used in Sec. 3.
 *
 * Conventions for every entry point:
 *  - Plain C types only. Pointers marked "device" must point to memory of the
 *    handle's CUDA device (cudaMalloc, torch CUDA tensors, managed memory);
 *    pointers marked "host" to host memory.
 *  - Every buffer is owned by the caller. xrd_pattern_batch allocates no
 *    memory: its scratch space is the caller's workspace.
 *  - Work is queued on the caller's stream and is asynchronous; outputs are
 *    valid after the stream has been synchronised. Calls on one handle must
 *    not run concurrently from several host threads.
 *  - Return value: XRD_OK or an error code. On error xrd_last_error() gives a
 *    one-line message. Data-dependent errors found on the device (an invalid
 *    cell, an atom with Z > zmax, a non-finite value, too little capacity) are
 *    reported per structure in xrd_pattern.status and summed in
 *    xrd_pattern.totals[3]; they never abort and never trap on the device.
 */
#ifndef XRD_H
#define XRD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XRD_OK 0
#define XRD_EINVAL 1    /* invalid argument, pointer, size or input value */
#define XRD_ECAPACITY 2 /* workspace or output capacity too small */
#define XRD_ECUDA 3     /* a CUDA call failed; see xrd_last_error */
#define XRD_ETIMEOUT 4  /* a bounded device-side wait ran out */

/* Precision of the structure-factor sum (Sec. 2, the structure-factor sum). */
#define XRD_FP64 0          /* every step in FP64 */
#define XRD_FP32_PHASE64 1  /* phase h.x+k.y+l.z formed and reduced mod 1 in FP64, the rest in FP32 */
#define XRD_FP32_PHASEFIX 2 /* coordinates in 32-bit fixed point, phase reduced mod 1 exactly in integers, the rest in FP32 */

typedef struct xrd_handle xrd_handle;

/* Batch of structures; every pointer is device memory, layouts are row-major. */
typedef struct {
    int32_t n_struct;        /* number of structures, >= 0 */
    int32_t zmax;            /* largest element number in coef, 0..255 */
    int64_t n_atoms;         /* total atoms = atom_off[n_struct] */
    const double* lattice;   /* [n_struct][6]: a, b, c (angstrom), alpha, beta, gamma (degrees) */
    const int64_t* atom_off; /* [n_struct + 1]: atoms of structure s are atom_off[s] .. atom_off[s+1]-1 */
    const double* frac;      /* [n_atoms][3]: fractional coordinates x, y, z */
    const int16_t* Z;        /* [n_atoms]: element number, 0..zmax */
    const double* occ;       /* [n_atoms]: site occupancy; a site shared by several species is one
                                record per species at the same coordinates */
    const double* B;         /* [n_atoms]: isotropic displacement (Debye-Waller) factor, angstrom^2 */
    const double* coef;      /* [zmax + 1][4][2]: (a_i, b_i) of f(s) = Z - 41.78214 s^2 sum a_i exp(-b_i s^2) */
} xrd_batch;

/* Smallest accepted merge tolerance, degrees. */
#define XRD_MIN_TT_TOL 1e-9

/* Options (host struct). */
typedef struct {
    double lambda;     /* wavelength, angstrom, > 0 */
    double tt_min;     /* 2-theta range in degrees, 0 <= tt_min < tt_max <= 180, both inclusive. The
                          Lorentz factor diverges at 180 degrees: a reflection within ~1e-6 degrees of it
                          gets a large finite factor that depends on the last bit of |g|^2. */
    double tt_max;
    double tt_tol;     /* merge tolerance in degrees, >= XRD_MIN_TT_TOL: join the peak while 2theta - anchor < tt_tol.
                          Smaller values are refused (XRD_EINVAL): 2theta itself carries ~1e-13 degrees of
                          rounding, and a reflection and its Friedel mate always share one peak. */
    double rel_cutoff; /* keep merged peaks with I > rel_cutoff * Imax; 0 keeps all; [0, 1) */
    int32_t scaled;    /* 1: scale intensities to 100 * (I / Imax); 0: absolute */
    int32_t precision; /* XRD_FP64, XRD_FP32_PHASE64 or XRD_FP32_PHASEFIX */
    int32_t tile;      /* structure-factor tile override: reflections per CTA, or -1 for the tuned value */
    int32_t reserved;  /* must be 0 */
} xrd_opts;

/* Sizes returned by xrd_query_sizes. */
typedef struct {
    int64_t n_refl;       /* Friedel-unique reflections of the whole batch (each stands for g and -g) */
    int64_t max_refl;     /* largest Friedel-unique count of one structure */
    int64_t n_tiles;      /* structure-factor tiles at the tuned tile size */
    size_t ws_bytes;      /* workspace bytes xrd_pattern_batch needs for this batch and these options */
    size_t ws_grad_bytes; /* workspace bytes xrd_pattern_broadened + xrd_pattern_grad need */
} xrd_sizes;

/* Uniform 2-theta grid of a broadened pattern: t_k = t0 + k dt, k = 0 .. n_pts - 1,
 * Gaussian peaks of full width at half maximum fwhm (degrees). */
typedef struct {
    double t0;        /* degrees */
    double dt;        /* degrees, > 0 */
    double fwhm;      /* degrees, > 0 */
    int32_t n_pts;    /* > 0 */
    int32_t reserved; /* must be 0 */
} xrd_grid;

/* Bit of xrd_pattern.flags: the cell is hexagonal (alpha, beta within 5 deg of
 * 90, gamma within 5 deg of 120, |a - b| < 0.01 A), so its families group the
 * Miller-Bravais indices (h, k, i = -h - k, l); (h, k, i, l) follows from hkl. */
#define XRD_FLAG_HEXAGONAL 1

/* Pattern output: device buffers owned by the caller. Peaks and families are
 * dense CSR arrays over the batch, in structure order; within a structure
 * peaks ascend in 2-theta. A capacity of n_refl (from xrd_query_sizes) is
 * always enough for both peaks and families. When a capacity is too small
 * every structure reports XRD_ECAPACITY, and totals[] says what was needed:
 * for a workspace too small, totals[0] is the reflection count it must hold
 * (xrd_query_sizes sizes it); for outputs too small, totals[0], totals[1]
 * and totals[2] are the reflections, peaks and families the outputs need.
 * The per-reflection list (refl_off != NULL) holds every Friedel-unique
 * reflection (first nonzero of h, k, l positive; each stands for g and -g,
 * which have the same intensity) before merging and cutoff, within a
 * structure in the order of the merge: ascending |g|^2, ties by descending
 * (h, k, l). Its capacity n_refl is enough. */
typedef struct {
    int64_t cap_peaks;  /* capacity of the per-peak arrays */
    int64_t cap_fam;    /* capacity of the per-family arrays */
    int64_t* peak_off;  /* [n_struct + 1]: peaks of structure s are peak_off[s] .. peak_off[s+1]-1 */
    double* two_theta;  /* [cap_peaks]: peak position, degrees (2-theta of the peak's first reflection) */
    double* intensity;  /* [cap_peaks]: merged intensity (scaled to 100 if opts.scaled) */
    double* d_hkl;      /* [cap_peaks]: d spacing of the peak's first reflection, angstrom */
    int64_t* fam_off;   /* [cap_peaks + 1]: families of global peak p are fam_off[p] .. fam_off[p+1]-1 */
    int32_t* hkl;       /* [cap_fam][3]: family representative (lexicographically largest member) */
    int32_t* mult;      /* [cap_fam]: family multiplicity (members over the full sphere). A family is
                           the reflections of a peak equal up to permutation and sign of (h, k, l); in a
                           hexagonal cell (alpha, beta within 5 deg of 90, gamma within 5 deg of 120,
                           |a - b| < 0.01 A) of the Miller-Bravais (h, k, i, l), i = -h - k, the 4-index
                           convention of the calculator the paper accelerates (Sec. 2) */
    int32_t* status;    /* [n_struct]: XRD_OK, XRD_EINVAL (bad cell or atom) or XRD_ECAPACITY */
    int64_t* totals;    /* [4]: reflections (Friedel-unique), peaks, families, structures with an error */
    int64_t cap_refl;   /* capacity of the per-reflection arrays (used when refl_off is not NULL) */
    int64_t* refl_off;  /* [n_struct + 1] or NULL: reflections of structure s are refl_off[s] .. refl_off[s+1]-1 */
    int32_t* refl_hkl;  /* [cap_refl][3]: (h, k, l) of each reflection */
    double* refl_tt;    /* [cap_refl]: its 2-theta, degrees */
    double* refl_I;     /* [cap_refl]: its intensity |F|^2 LP, unscaled and unmerged (that of g, and of -g) */
    int32_t* flags;     /* [n_struct] or NULL: per-structure flag bits (XRD_FLAG_HEXAGONAL) */
} xrd_pattern;

/*
 * Create a handle bound to CUDA device `device`. Returns XRD_OK or
 * XRD_ECUDA/XRD_EINVAL. The handle owns eight non-blocking side streams: the
 * nine post-processing size classes of xrd_pattern_batch (the largest as flat
 * device-wide passes) run on them and the caller's stream concurrently,
 * forked from and joined back into the caller's stream by events (so a
 * capture of the call on the caller's stream takes them in as branches).
 */
int xrd_create(xrd_handle** h, int device);
/* Destroy a handle (NULL is ignored). */
void xrd_destroy(xrd_handle* h);
/* Message of the last error on this handle ("" if none); valid until the next call. */
const char* xrd_last_error(const xrd_handle* h);

/*
 * Count the reflections of a batch (Sec. 2: the reciprocal-lattice points
 * inside the sphere the 2-theta range reaches) and size the workspace.
 * Runs the enumeration count on `stream` and synchronises it. May allocate
 * device memory owned by the handle (never on the hot path). Per-structure
 * input errors are not reported here; xrd_pattern_batch reports them.
 */
int xrd_query_sizes(xrd_handle* h, const xrd_batch* batch, const xrd_opts* opts, xrd_sizes* sizes,
                    void* stream /* cudaStream_t */);

/*
 * Accuracy of the FP32 variants. The agreement the paper quotes is per peak
 * (Sec. 3: peak intensities relative to the largest, positions); the FP32
 * variants hold every kept peak's intensity to 1e-5 of itself. The FP32 pass
 * errs by about 1.5e-7 of sqrt(sum_j a_j^2) in F (a_j = occ_j exp(-B_j s^2)
 * max(|f_j|, Z_j)), so a weak reflection, one whose atoms nearly cancel, has a
 * large relative error. The call therefore re-evaluates, in double-float
 * arithmetic (about 48 bits, from exact 64-bit fixed-point phases), every
 * reflection whose 3-sigma error bound exceeds 4e-6 of max(I, c M) (M the
 * structure's largest reflection intensity, c the cutoff fraction, 1e-3 when
 * the cutoff is off): typically a few percent of the reflections.
 * xrd_set_refine(h, 0) turns this off (a diagnostic: the FP32 pass alone).
 */
int xrd_set_refine(xrd_handle* h, int enabled);

/*
 * Friedel-unique reflection count of every structure (Sec. 2: the
 * reciprocal-lattice points inside the sphere the 2-theta range reaches, one
 * per pair g, -g): counts is a host array of n_struct. Runs the enumeration
 * count on `stream` and synchronises it; may allocate device memory owned by
 * the handle (never on the hot path). With the atom counts it gives each
 * structure's structure-factor cost, R x N, which the multi-GPU path balances
 * across ranks. An invalid cell counts 0.
 */
int xrd_reflection_counts(xrd_handle* h, const xrd_batch* batch, const xrd_opts* opts, int64_t* counts,
                          void* stream /* cudaStream_t */);

/*
 * The whole pattern of every structure (Sec. 2 steps, then Sec. 2's optional
 * cutoff and Sec. 3's 0-100 scale): enumerate the Friedel-unique reflections
 * with r_min <= |g| <= r_max, evaluate F(g) = sum_j occ_j f_j(s)
 * exp(-B_j s^2) exp(2 pi i g.x_j) and I = |F|^2 LP, sort by 2-theta, merge
 * reflections within tt_tol of a peak's first reflection, group them into
 * families equal up to permutation and sign of (h, k, l), apply the cutoff
 * and scale. `workspace` is device memory of at least sizes.ws_bytes (from
 * xrd_query_sizes with the same batch and options), 256-byte aligned. No
 * allocation, no host synchronisation: the call can be captured in a CUDA
 * graph. Errors found on the device are reported in out->status/out->totals.
 */
int xrd_pattern_batch(xrd_handle* h, const xrd_batch* batch, const xrd_opts* opts, const xrd_pattern* out,
                      void* workspace, size_t ws_bytes, void* stream /* cudaStream_t */);

/*
 * Gaussian-broadened pattern of every structure (the differentiable profile
 * used for refinement and for generating training patterns with peak
 * broadening; Sec. 1 motivates both):
 *   y[s][k] = sum over reflections g of structure s in the 2-theta range of
 *             I_g exp(-(t_k - 2theta_g)^2 / (2 sigma^2)),  sigma = fwhm / (2 sqrt(2 ln 2)),
 * with I_g = |F(g)|^2 LP unscaled and unmerged (g and -g both counted), each
 * Gaussian cut at |t_k - 2theta_g| <= about 6 sigma (grid points b - W .. b + W + 1
 * around the grid cell b of 2theta_g, W = ceil(6 sigma / dt); the cut changes y by
 * less than 2e-8 of a peak). opts.precision must be XRD_FP32_PHASEFIX;
 * rel_cutoff, scaled and tt_tol do not enter the result (they are validated as
 * for xrd_pattern_batch). y is device float [n_struct][n_pts].
 * status (device [n_struct]) and totals (device [4]) as in xrd_pattern. The
 * workspace (>= sizes.ws_grad_bytes) keeps the reflection list, F and dF/ds^2
 * for xrd_pattern_grad: pass the same workspace, unmodified, to that call.
 */
int xrd_pattern_broadened(xrd_handle* h, const xrd_batch* batch, const xrd_opts* opts, const xrd_grid* grid,
                          float* y, int32_t* status, int64_t* totals, void* workspace, size_t ws_bytes,
                          void* stream /* cudaStream_t */);

/*
 * Gradient of a loss L through the broadened pattern of the preceding
 * xrd_pattern_broadened call (same batch, options, grid and workspace), given
 * dL_dy (device float [n_struct][n_pts]): writes d_frac (device float
 * [n_atoms][3], dL/dx per fractional unit), d_B (device float [n_atoms],
 * per angstrom^2) and d_lattice (device float [n_struct][6]: dL/da, dL/db,
 * dL/dc per angstrom, dL/dalpha, dL/dbeta, dL/dgamma per degree). The
 * reflection set is the one enumerated by the forward call, held fixed.
 * Structures with a non-OK status get zero gradients.
 */
int xrd_pattern_grad(xrd_handle* h, const xrd_batch* batch, const xrd_opts* opts, const xrd_grid* grid,
                     const float* dL_dy, float* d_frac, float* d_B, float* d_lattice, void* workspace,
                     size_t ws_bytes, void* stream /* cudaStream_t */);

/*
 * Experimental effects of an augmented pattern (Sec. 1: synthetic training
 * patterns for ML models carry peak broadening, noise and preferred
 * orientation), one set per structure. Every pointer is a device array owned
 * by the caller and read during the call only.
 */
typedef struct {
    const double* fwhm;        /* [n_struct] pseudo-Voigt FWHM, degrees: 0 < fwhm <= 1e6 and 2 dt / fwhm <= 1e6 */
    const double* eta;         /* [n_struct] Lorentzian fraction, 0 <= eta <= 1 */
    const double* po_dir;      /* [n_struct][3] preferred-orientation direction, reciprocal-lattice components
                                  (not zero), or NULL: no preferred orientation */
    const double* po_r;        /* [n_struct] March-Dollase r, 1e-6 <= r <= 1e6; NULL exactly when po_dir is */
    const float* noise_z;      /* [n_struct][n_pts] standard normal draws, or NULL: no noise */
    const double* noise_sigma; /* [n_struct] noise scale >= 0; NULL exactly when noise_z is */
} xrd_augment;

/*
 * Augmented pattern of every structure on the grid t_k = t0 + k dt:
 *   y[s][k] = sum over reflections g of structure s in the 2-theta range
 *             (g and -g both counted, unmerged, no cutoff) of
 *             |F(g)|^2 LP P(g) PV(t_k - 2theta_g),
 *   P(g)  = (r^2 cos^2 a + sin^2 a / r)^(-3/2)   (March-Dollase; a = angle between g
 *           and po_dir in the reciprocal metric; P = 1 without po_dir),
 *   PV(u) = eta (2 / (pi w)) / (1 + x^2) + (1 - eta) (2 / w) sqrt(ln 2 / pi) 2^(-x^2),
 *           x = 2 u / w, w = fwhm (area-normalised pseudo-Voigt),
 * then, with noise_z, y[s][k] += sigma sqrt(max(y[s][k], 0)) z[s][k]. The
 * Lorentzian is summed over every grid point (no window); a reflection's
 * Gaussian is skipped only on runs of 256 consecutive grid points where it
 * stays below 2^-40 of its peak (x^2 >= 40). grid.fwhm is ignored; grid.n_pts <= 2^22
 * and every 2-theta in [tt_min, tt_max] lies within 2^22 dt of t0.
 * opts.precision must be XRD_FP32_PHASEFIX; rel_cutoff, scaled and tt_tol do
 * not enter the result (they are validated as for xrd_pattern_batch). y is
 * device float [n_struct][n_pts]; status and totals as in
 * xrd_pattern_broadened. A structure whose effect parameters break the rules
 * of xrd_augment gets status XRD_EINVAL and a zero row, and counts in
 * totals[3]. Workspace as xrd_pattern_broadened (>= sizes.ws_grad_bytes); the
 * call overwrites the state a following xrd_pattern_grad would need.
 * Returns XRD_EINVAL for NULL or inconsistent pointers and an invalid grid.
 */
int xrd_pattern_augmented(xrd_handle* h, const xrd_batch* batch, const xrd_opts* opts, const xrd_grid* grid,
                          const xrd_augment* aug, float* y, int32_t* status, int64_t* totals, void* workspace,
                          size_t ws_bytes, void* stream /* cudaStream_t */);

/*
 * Launch-shape tuning of the structure-factor kernel (the batching pattern of
 * the engine: thousands of uneven structures in one persistent launch). Runs
 * xrd_pattern_batch (same arguments) with each shape -- 2 or 4 reflections per
 * lane (warp tiles of 64 or 128 reflections) and, for XRD_FP32_PHASEFIX, 1, 2
 * or 4 warps per CTA, and lanes taking either 4 strided reflections or one run
 * of up to 4 reflections consecutive in l (one sin/cos pair per run and atom,
 * the phase factor then rotated from l to l + 1; the enumeration builds the
 * runs) -- times the stages a shape changes (count, scan, emit, structure
 * factor; the minimum of four calls) with CUDA events, synchronising `stream`,
 * and keeps the fastest shape in the handle, then picks the enumeration
 * kernels' launch shape (xrd_set_enum_threads) the same way; later calls with opts.tile = -1 use
 * it. Writes the chosen tile, warps and runs (0 or 1) if the pointers are not
 * NULL. Returns after `stream` has been synchronised (every tuning call has
 * finished). Not capturable.
 */
int xrd_autotune(xrd_handle* h, const xrd_batch* batch, const xrd_opts* opts, const xrd_pattern* out,
                 void* workspace, size_t ws_bytes, void* stream /* cudaStream_t */, int32_t* best_tile,
                 int32_t* best_warps, int32_t* best_runs);

/*
 * Work of the structure-factor stage of the last xrd_pattern_batch call on
 * this workspace (same batch): counts[0] = terms to evaluate (Friedel-unique
 * reflection x atom), counts[1] = phase-factor seeds (one sin/cos pair per term
 * with strided tiles, per run and atom with runs consecutive in l), counts[2] =
 * structure-factor tiles, counts[3] = reflections re-evaluated in double-float
 * (FP32 variants). Host array of 4. Reduces the workspace's per-structure counts on
 * `stream` (one small kernel) and synchronises it. These counts set the SFU time floor of the
 * batch (the paper has no counterpart; it is for the roofline of the kernel).
 */
int xrd_work_counts(xrd_handle* h, const xrd_batch* batch, const void* workspace, void* stream /* cudaStream_t */,
                    int64_t* counts);

/*
 * Issue rates of the units that bound the structure-factor kernel, measured on
 * the handle's device (the paper has no counterpart: these are the peak of the
 * kernel's roofline). rates[0..4] = MUFU sin, MUFU cos, MUFU ex2, FP32 FMA and
 * FP64 FMA operations per SM per clock (host array of 5): one CTA of 1024
 * threads with eight independent chains of the operation per thread, timed by
 * the SM's clock64 counter. Allocates a few bytes of device memory and
 * synchronises; not for the hot path.
 */
int xrd_unit_rates(xrd_handle* h, double* rates);

/* Set the structure-factor launch shape directly (tile 64 or 128 reflections per
 * warp, 1, 2 or 4 warps per CTA; warps apply to XRD_FP32_PHASEFIX; runs = 1,
 * with tile 128 and XRD_FP32_PHASEFIX only, makes lanes take runs consecutive in l). */
int xrd_set_sf_shape(xrd_handle* h, int tile, int warps, int runs);

/*
 * Symmetry-aware family mode (the calculator interface of Sec. 2 groups the
 * equivalent reflections of a peak into families): with n_ops > 0, the
 * reflections of a merged peak are grouped by their orbits under the given
 * point group instead of by permutation and sign of (h, k, l) (or of
 * (h, k, i, l) for a hexagonal cell). ops: host array [n_ops][3][3] of
 * integer matrices M acting on (h, k, l) as a column vector, entries -1, 0 or
 * 1, n_ops <= 48 (any generating set's closure, e.g. the 48 operations of
 * m-3m; Friedel's law adds the inversion by itself). The family of g is
 * {M g, -M g}; its representative is still the lexicographically largest
 * member present in the peak, and its multiplicity the number of members over
 * the full sphere. For a structure with that symmetry, the multiplicities are
 * the orbit sizes of International Tables. The operations are copied
 * (synchronously) to the handle's device; n_ops = 0 restores the default. The
 * mode applies to later xrd_query_sizes and xrd_pattern_batch calls on the
 * handle (its workspace holds 16 more bytes per reflection) and adds two kernel
 * launches per call.
 */
int xrd_set_point_group(xrd_handle* h, const int32_t* ops, int n_ops);

/* Launch shape of the enumeration kernels (256 by default): 64, 128 or 256 threads per CTA
 * with one warp per structure (the CTA's whole block takes the few structures above 1024
 * columns or 4096 reflections), or 512 or 1024 threads with one CTA per structure.
 * Neither the order of the enumerated reflections nor the pattern changes with it. */
int xrd_set_enum_threads(xrd_handle* h, int threads);

/* Test hook of the bounded device-side wait. The flat post-processing passes of
 * structures above 6144 reflections run as one cooperative kernel whose passes
 * are separated by a grid-wide barrier; each wait there is bounded to about one
 * second, after which that kernel's structures report XRD_ETIMEOUT (no peaks)
 * and the call completes. extra > 0 makes the barrier wait for `extra` arrivals
 * that never come, so that the bound is exercised on purpose; 0 (the default)
 * restores normal operation. XRD_EINVAL for extra < 0 or > 1024. */
int xrd_test_flat_barrier(xrd_handle* h, int extra);

/*
 * CUDA graph of one xrd_pattern_batch call with exactly these arguments (the
 * device buffers are baked into the graph: replays read the batch's current
 * contents and rewrite the outputs). xrd_graph_create synchronises the device
 * (earlier work on these buffers must be finished), runs one eager call on a
 * private stream, synchronises it, then captures a second call; *graph gets an
 * opaque executable. xrd_graph_launch replays it on `stream`;
 * xrd_graph_destroy frees it. The batch's sizes (and so the workspace) must
 * not grow between replays.
 */
int xrd_graph_create(xrd_handle* h, const xrd_batch* batch, const xrd_opts* opts, const xrd_pattern* out,
                     void* workspace, size_t ws_bytes, void** graph);
int xrd_graph_launch(xrd_handle* h, void* graph, void* stream /* cudaStream_t */);
void xrd_graph_destroy(void* graph);

/* Stage timing. Mode 1: xrd_pattern_batch records CUDA events between all
 * stages on its stream; mode 2: only around the structure-factor stage (each
 * event is a node of a captured graph and costs time, so mode 2 perturbs a
 * timed run least); 0: off (XRD_EINVAL for another value). xrd_stage_times
 * synchronises on the last event of the last recorded call and writes up to n
 * stage durations in milliseconds (order: prep, atoms, count, scan, emit,
 * structure factor, refine, post, compact, profile sum; in mode 2 every stage but the
 * structure factor reads 0; after an xrd_pattern_augmented call, in either
 * mode, only the profile sum -- the two kernels after the structure factors --
 * is timed and the others read 0) and returns the count. */
int xrd_set_profiling(xrd_handle* h, int enabled);
int xrd_stage_times(xrd_handle* h, float* ms, int n);

/*
 * Allocation-free variant of xrd_pattern_batch (the paper has no counterpart:
 * it is an interface for callers that may not allocate device memory, such as
 * code running under a framework-owned memory pool, plug-ins whose host forbids
 * cudaMalloc, or loops where an allocation's implicit synchronisation is not
 * acceptable). It computes exactly what xrd_pattern_batch computes, with the
 * same inputs and caller-owned outputs, but its scratch space is a fixed
 * file-scope device array of XRD_NOALLOC_SCRATCH_BYTES instead of a workspace.
 *  - Nothing is allocated by the call: no cudaMalloc, no cudaFree, no
 *    allocating library routine.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, which may load the module); make that first call
 *    before any stream capture on that device. The address is cached with the
 *    ID of the context it belongs to and looked up again when the device's
 *    context changes (after cudaDeviceReset, say); make the first call after
 *    such a change before any stream capture too.
 *  - When the array is reserved depends on CUDA's module loading: with lazy
 *    loading (the default) on a device the first time this entry point runs
 *    there; with eager loading (CUDA_MODULE_LOADING=EAGER) on every device
 *    where the library is loaded, called there or not. It stays reserved
 *    until the process exits.
 *  - Limit: the per-structure and per-atom arrays (about 250 bytes per
 *    structure and 120 bytes per atom) plus about 105 bytes per Friedel-unique
 *    reflection must fit in 64 MiB. A batch whose per-structure and per-atom
 *    part does not fit is rejected on the host with XRD_ECAPACITY; one whose
 *    reflections do not fit is flagged on the device (status XRD_ECAPACITY for
 *    every structure, totals[3] = n_struct), as with a short workspace.
 *  - All calls share the array and it keeps the last call's contents; the call
 *    clears what must start at zero. Calls that overlap on the GPU (several
 *    streams or host threads at once) race on it: serialise them.
 */
#define XRD_NOALLOC_SCRATCH_BYTES (64u << 20)
int xrd_pattern_batch_noalloc(xrd_handle* h, const xrd_batch* batch, const xrd_opts* opts, const xrd_pattern* out,
                              void* stream /* cudaStream_t */);

#ifdef __cplusplus
}
#endif
#endif /* XRD_H */
