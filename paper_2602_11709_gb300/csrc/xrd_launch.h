// Host-side launch arguments shared by the C ABI layer and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "xrd_internal.cuh"

namespace xrd {

struct GeomArgs {
    int n_struct, zmax, rb;  // rb: reflections a structure-factor lane takes (2 or 4)
    int runs_mode;           // 1: tiles of 32 runs of <= rb reflections consecutive in l; 0: tiles of 32 rb reflections
    int enum_threads;        // threads per structure of k_count / k_emit (64, 128 or 256; the same for both)
    int64_t n_atoms;
    double r2min, r2max, rmax;
    int64_t cap_refl;
    const double* lattice;
    const int64_t* atom_off;
    const double* frac;
    const int16_t* Z;
    const double* occ;
    const double* B;
    const double* coef;
    Geo* geo;
    Coef32* coef32;
    Atom32* atom32;
    Atom64* atom64;
    float2* astep;   // [atoms] exp(2 pi i z) of each element-sorted atom
    int64_t* refl_cnt;
    int64_t* run_cnt;  // [n_struct] runs of each structure
    int* runs;       // [reflections] run entries (first reflection within the structure << 3 | length)
    unsigned long long* work;  // [3] structure-factor work: terms, phase-factor seeds, tiles (k_scan_refl)
    int64_t* refl_off;
    int* tile_off;   // [n_struct + 1] first structure-factor tile of each structure; [n_struct] = tiles
    int* order;      // [n_struct] structures by atom count, largest first
    int2* tile_tab;  // [tiles] (structure, first reflection) of each structure-factor tile
    int* atom_bad;   // [n_struct] 1 where an atom of the structure is invalid
    int atoms_set_geo;  // k_atoms also marks such structures invalid in geo (only when it runs before k_count)
    int* cls_list;   // [kPostClasses][n_struct] post-processing size classes (nullptr: not built)
    int* abort_flag; // flags[0]; flags[1] output abort, flags[2] tile queue, flags[4..6] flat-pass grid barrier, flags[26..28] enumeration
                     // claims, flags[kFlagClsCnt + c] class counts, flags[kFlagClsNext + c] class work counters
    int64_t* totals;
    int32_t* status;
    double* q;
    uint32_t* key;
    long long* parts;  // chunk sums of the multi-block scan (nullptr: single-block scan)
    int* oparts;       // [chunks][4096] bin counts of the multi-block order (nullptr: one-block order)
    int* enum_ctr;     // flags[26..28]: structure claims of counting, of emission's warps and of its CTAs
    const float4* sctab;  // [256] cos and sin of 2 pi k / 256 as two floats (the re-evaluation's table)
    unsigned* imax;    // [n_struct] largest reflection intensity slot, zeroed by k_prep (or nullptr)
    int32_t* out_flags;  // [n_struct] caller's flag words, written by k_prep (or nullptr)
    float4* cdd;       // [(zmax + 1) * 4] (a, b) coefficients as two floats, by k_coef (or nullptr)
    AtomR* atomr;      // [atoms] records of the accurate re-evaluation, by k_atoms (or nullptr)
};

struct SfArgs {
    int n_struct, precision, tile, grid, zmax;
    int rb, warps;  // launch shape: reflections per lane (2 or 4), warps per CTA (1, 2 or 4)
    int runs_mode;  // lanes take runs (integer phase only) instead of strided reflections
    double lambda;
    const int64_t* atom_off;
    const int64_t* refl_off;
    const int* tile_off;  // [n_struct + 1]: [n_struct] is the number of tiles
    const int2* tile_tab; // [tiles] (structure, first run or reflection within it), largest-first order
    const int64_t* run_cnt;  // [n_struct] runs of each structure
    const int* runs;      // [reflections] run entries, indexed from refl_off[s]
    const float2* astep;  // [atoms] exp(2 pi i z) of each element-sorted atom (the l + 1 step)
    int* tile_counter;    // work-queue head, zeroed by the caller
    const int* abort_flag;
    const Coef32* coef32;
    const double* coef;
    const Atom32* atom32;
    const Atom64* atom64;
    const double* q;
    const uint32_t* key;
    double* I;   // per reflection intensity |F|^2 LP (one Friedel half-space member), XRD_FP64
    float* If;   // the same in FP32 for the FP32 variants
    float2* F;   // optional per-reflection F (nullptr: not stored)
    float4* Fx;  // gradient path: (Re F, Im F, Re dF/ds^2, Im dF/ds^2) per reflection (nullptr otherwise)
    float* Ig;   // gradient path: |F|^2 LP per reflection
    float* Eb;   // FP32 pattern variants: bound of the intensity's rounding error per reflection (or nullptr):
                 // LP dF (2 |F| + dF) with dF = eps_k sqrt(sum_j a_j^2), a_j = occ DW max(|f|, Z)
    int* Es;     // the structure of each reflection whose bound exceeds tau times its intensity (others: unset)
    float eps_k; // K times the relative error of one FP32 term (the bound of |dF| / sqrt(sum a_j^2))
    float tau;
    unsigned* imax;  // FP32 pattern variants: [n_struct] bits of the largest reflection intensity (zeroed by k_prep)
};

// Device tables of the accurate re-evaluation (built once per handle).
struct RefineTables {
    const float4* sc;  // [256] cos and sin of 2 pi k / 256, two floats each
    const float2* ex;  // [64] 2^(-j / 64) as two floats
};

struct RefineArgs {
    int n_struct, zmax, grid;  // grid = number of SMs
    double lambda;
    float l2f;       // lambda^2 / 4
    float l2h, l2l;  // lambda^2 / 4 as two floats
    float tau;    // intensity error allowed without re-evaluation, relative to max(I, cref M)
    float cref;   // cutoff fraction (the floor of the guarantee), relative to the largest reflection M
    const int* abort_flag;
    unsigned long long* nref;     // reflections re-evaluated: the candidate list's length (zeroed per call)
    int64_t* cand_r;              // [reflections] candidate list: reflection index
    int* cand_s;                  // [reflections] and its structure
    const int64_t* refl_off;
    const int64_t* atom_off;
    const double* q;
    const uint32_t* key;
    float* If;          // FP32 intensities, rewritten for the re-evaluated reflections
    const float* Eb;    // bound of the FP32 intensity's rounding error per reflection (k_sf)
    const int* Es;      // the reflection's structure where Eb > tau If (k_sf)
    const unsigned* imax;  // largest intensity of each structure (bits)
    const AtomR* atomr;
    const float4* cdd;
    const float4* sc;
    const float2* ex;
    const int* atom_bad;
};

// A reflection record of the flat post passes: one 16-byte load or store.
struct __align__(16) PfRec {
    double q;
    uint32_t key;
    float I;
};

struct PostArgs {
    int n_struct, scaled, grid;  // grid = number of SMs
    double lambda, tol, cutoff, r2min, r2max;
    double l2d;                          // lambda^2 / 4
    const TTab* ttab;                    // 2-theta table (device)
    float ttol, lo3, hi3, l2f, lhf;      // FP32: tan(tol / 4) (tol in radians), r2min^1.5, r2max^1.5, lambda^2/4, lambda/2
    const Geo* geo;     // per structure: the hexagonal flag picks the family grouping
    const int64_t* refl_off;
    const int* abort_flag;
    const double* q;
    const uint32_t* key;
    const double* I;    // FP64 intensities (XRD_FP64), or
    const float* If;    // FP32 intensities (the FP32 variants)
    const int* cls_list;  // [kPostClasses][n_struct] structures of each size class, largest first
    const int* cls_cnt;   // [kPostClasses]
    int* cls_next;        // [kPostClasses] work counters (zero at launch)
    // scratch of the flat passes of the largest class (indexed by reflection)
    int* g_bkt;   // n_refl + n_struct entries
    uint8_t* g_flag;
    int* g_pstart;
    double* g_psum;
    int* g_fcnt;
    // staging of kept peaks and families (indexed by reflection offset)
    double* st_q;      // anchor |g|^2 of each kept peak
    double* st_I;      // its intensity: FP64, or FP32 (first half) in the FP32 variants
    int* st_foff;
    uint32_t* st_key;  // packed hkl of each family's representative
    int* st_mult;
    int64_t* npk;  // kept peaks per structure
    int64_t* nfm;  // families of kept peaks per structure
    // structures with an invalid atom: no peaks, status XRD_EINVAL (counted in totals[3])
    const int* atom_bad;
    int32_t* status;
    int64_t* totals;
    // the caller's per-reflection list in merge order (refl_hkl nullptr: not written)
    int64_t cap_refl;
    int32_t* refl_hkl;
    double* refl_tt;
    double* refl_I;
    float l2h, l2l;  // lambda^2 / 4 as two floats (2-theta of the list)
    // the flat passes of the largest class (k_post_flat.cu)
    int* pf_bar;                   // flags[kFlagPfBar..+2]: grid barrier of the flat passes (zero at launch)
    int pf_bar_extra;              // arrivals the barrier also waits for (a test of its bounded wait; 0)
    int* pf_voff;                  // [n_struct + 1] virtual offsets of the class's structures
    unsigned long long* pf_smax;   // [n_struct] bits of each structure's largest peak sum
    int* pf_scal;                  // [4]: reflections of the class (V), its peaks
    long long* pf_parts;           // [2 kPfScanBlocksMax] segment sums of the scans
    int* pf_pst;                   // [reflections + 1] peak starts, then peak ids
    int* pf_pj;                    // [reflections] structure (class-list position) of each peak
    int* pf_kidx;                  // [reflections + 1] kept-peak index of each peak
    int* pf_fidx;                  // [reflections + 1] family offset of each peak
    PfRec* pf_rec;                 // [reflections] (|g|^2, key, FP32 intensity) records, bucket then sorted order
    double* pf_rI;                 // [reflections] FP64 intensities beside them (the FP64 variant)
    // the symmetry-aware family mode: the caller's point group (nullptr, 0: permutation and sign)
    const int8_t* pg;              // [npg][3][3] operations on (h, k, l), entries in {-1, 0, 1}
    int npg;
    const unsigned long long* fkg; // [reflections] family key of every reflection under pg (or nullptr)
    unsigned long long* pf_sfk;    // [reflections] the same for the sorted records of the flat passes
};
constexpr int kMaxPgOps = 48;
void launch_pg_keys(const PostArgs& a, unsigned long long* fkg, cudaStream_t st);
constexpr int kPfScanBlocksMax = 1024;

struct CompactArgs {
    int n_struct, grid;  // grid = number of SMs
    int64_t cap_peaks, cap_fam;
    const int64_t* refl_off;
    const int* abort_flag;
    const int64_t* npk;
    const int64_t* nfm;
    int64_t* fam_soff;  // [n_struct + 1] scratch: exclusive scan of nfm
    const double* st_q;
    const double* st_I;
    float l2h, l2l;        // lambda^2 / 4 as two floats
    const TTab* ttab;      // 2-theta table
    const int* st_foff;
    const uint32_t* st_key;
    const int* st_mult;
    int fi;             // st_I holds FP32 intensities
    int* out_abort;     // set when the output capacity is too small
    long long* parts;   // chunk sums of the multi-block scan (nullptr: single-block scan)
    xrd_pattern out;
};

struct GradArgs {
    int n_struct, n_pts, W;
    int64_t n_atoms;
    double t0, dt, sigma, l2d;
    float l2h, l2l;  // lambda^2 / 4 as two floats
    const TTab* ttab;
    const Geo* geo;
    const double* lattice;
    const int64_t* refl_off;
    const int64_t* atom_off;
    const int* abort_flag;
    const double* q;
    const uint32_t* key;
    const float4* Fx;  // (Re F, Im F, Re dF/ds^2, Im dF/ds^2)
    const float* Ig;   // |F|^2 LP
    int* tb;           // grid cell of each reflection's 2theta (INT_MIN: off the grid)
    float* td;         // position within the cell, [0, 1)
    int* perm;         // per-reflection scratch
    float* y;          // [n_struct][n_pts]
    const float* dLdy; // [n_struct][n_pts]
    float* U;          // dL/dI LP Re F per reflection
    float* V;          // dL/dI LP Im F
    const Atom32* atom32;
    const Coef32* coef32;
    float* d_frac;
    float* d_B;
    float* d_lat;
};

struct AugArgs {
    int n_struct, n_pts;
    double t0, dt, inv_dt;
    float l2h, l2l;  // lambda^2 / 4 as two floats
    const TTab* ttab;
    const Geo* geo;
    const int64_t* refl_off;
    const int* abort_flag;
    const double* q;
    const uint32_t* key;
    const float* Ig;  // |F|^2 LP per reflection (one Friedel member)
    // effect parameters (device, per structure; po_* and noise_* may be nullptr)
    const double* fwhm;
    const double* eta;
    const double* po_dir;
    const double* po_r;
    const float* noise_z;
    const double* noise_sigma;
    int* aorder; // [n_struct] structures by reflection count, largest first
    int32_t* status;
    int64_t* totals;
    float* y;    // [n_struct][n_pts]
};

// pdl: launch as a programmatic dependent of the previous kernel on st (only
// when that kernel directly precedes it on the stream)
void launch_prep(const GeomArgs& a, cudaStream_t st, bool pdl);
void launch_coef(const GeomArgs& a, cudaStream_t st, bool pdl);
void launch_atoms(const GeomArgs& a, cudaStream_t st, bool pdl);
void launch_order(const GeomArgs& a, cudaStream_t st, bool pdl);
size_t order_parts_bytes(int64_t n);  // bytes of GeomArgs::oparts for n structures (0: one-block order)
void launch_count(const GeomArgs& a, cudaStream_t st, bool pdl);
void launch_count_only(const GeomArgs& a, cudaStream_t st);
void launch_scan_refl(const GeomArgs& a, cudaStream_t st, bool pdl);
void launch_work(const GeomArgs& a, unsigned long long* out, cudaStream_t st);  // out: device [3], zeroed
void launch_emit(const GeomArgs& a, cudaStream_t st, bool pdl);
void launch_sf(const SfArgs& a, cudaStream_t st, bool pdl);
RefineTables init_refine_tables(cudaStream_t st);  // fills the tables, returns their device addresses
void launch_refine(const RefineArgs& a, cudaStream_t st, bool pdl);
size_t post_smem_bytes(int cap);
void launch_post_flat(const PostArgs& a, int cls, cudaStream_t st);
void launch_post(const PostArgs& a, const cudaStream_t* st);  // st[kPostStreams]: a stream per class
void launch_compact(const CompactArgs& a, cudaStream_t st);
const TTab* init_tables(cudaStream_t st);  // fills the 2-theta table, returns its device address
size_t broaden_smem_bytes(int n_pts, int W);
void launch_broaden(const GradArgs& a, cudaStream_t st);
void launch_grad(const GradArgs& a, cudaStream_t st);
void launch_aug(const AugArgs& a, cudaStream_t st);   // per-reflection amplitudes, then the profile sums

// handle accessors for entry points defined outside api.cu
int handle_device(const xrd_handle* h);
int set_error(xrd_handle* h, int code, const char* msg);

}  // namespace xrd
