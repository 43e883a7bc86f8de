// C ABI of the powder-XRD engine: handles, argument validation, workspace
// layout and the launch sequence of one pattern batch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "xrd_launch.h"

constexpr int kEvents = 12;

struct xrd_handle {
    int device = 0;
    int sms = 0;
    std::string err;
    int profiling = 0;  // 0 off, 1 every stage, 2 the structure-factor stage only
    int recorded = 0;   // the mode of the last recorded call (3: an augmented-pattern call)
    cudaEvent_t ev[kEvents] = {};  // stage boundaries; the last two bracket the augmented profile sum
    void* qbuf = nullptr;  // query scratch owned by the handle
    size_t qbuf_bytes = 0;
    const xrd::TTab* ttab = nullptr;  // 2-theta table on the handle's device
    int sf_rb = 4, sf_warps = 2;        // structure-factor launch shape (xrd_autotune)
    int sf_runs = 0;                    // lanes take runs consecutive in l (integer phase only)
    int enum_threads = 256;             // threads per structure of the enumeration kernels (xrd_autotune)
    // side streams for the concurrent post-processing size classes (fork/join by events)
    cudaStream_t side[xrd::kPostStreams - 1] = {};
    cudaEvent_t fork = nullptr, join[xrd::kPostStreams - 1] = {};
    // the input-only front (coefficients, atom packing, largest-first order) runs on side[0]
    // beside the enumeration: forked by front, joined by order_done and atoms_done
    cudaEvent_t front = nullptr, order_done = nullptr, atoms_done = nullptr;
    unsigned long long* wbuf = nullptr;  // device [3]: xrd_work_counts result
    xrd::RefineTables rtab{};            // tables of the accurate re-evaluation on the handle's device
    int8_t* pg = nullptr;                // device [kMaxPgOps][9]: the point group of the family mode
    int npg = 0;                         // its operations (0: families by permutation and sign)
    int refine = 1;                      // re-evaluate weak reflections of the FP32 variants (xrd_set_refine)
    int bar_extra = 0;                   // xrd_test_flat_barrier: arrivals the flat passes' barrier waits for in vain
};

namespace {

constexpr int kRunsPerTileHost = xrd::kRunsPerTile;  // structure-factor tile: 32 runs (one per lane)
// flags area, zeroed at the start of every call: flag words (see GeomArgs::abort_flag), the
// structure-factor work counters (3 x 64 bit) at byte kWorkOffset, the re-evaluation's
// reflection count (64 bit) at kRefinedOffset, the enumeration claims at int 26 and the post
// class counts and work counters at ints kFlagClsCnt and kFlagClsNext
constexpr int kFlagBytes = 256;
constexpr int kWorkOffset = 64;
constexpr int kRefinedOffset = 96;
constexpr int kStages = 9;
constexpr int kSfStage = 5;      // index of the structure-factor stage
constexpr int kRefineStage = 6;  // index of the re-evaluation stage
// Re-evaluation of weak reflections (FP32 variants): the bound of |dF| / sqrt(sum a_j^2) of the FP32
// pass, about 4 times its measured RMS error (9e-8 with sin/cos on the FMA pipe, every precision
// variant and launch shape), and the error allowed without re-evaluation
constexpr float kRefineEpsK = 3.5e-7f;
constexpr float kRefineTau = 4e-6f;
constexpr double kRefineFloorNoCut = 1e-3;  // guarantee floor (fraction of the largest) with the cutoff off

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int fail(xrd_handle* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    return code;
}

int cuda_fail(xrd_handle* h, cudaError_t e, const char* where)
{
    return fail(h, XRD_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// Byte offsets of every array in the caller's workspace.
struct Layout {
    size_t geo, refl_cnt, run_cnt, refl_off, tile_off, order, atom_bad, cls_list, tile_tab, npk, nfm, fam_soff,
        flags, coef32, atom32, atom64, astep, imax, cdd, atomr;
    size_t q, key, runs, I, Eb, cand_r, cand_s, g_bkt, g_flag, g_pstart, g_psum, g_fcnt;
    size_t st_q, st_I, st_foff, st_key, st_mult;
    size_t parts, oparts, pf, pf_rec, fkg, pf_sfk;
    size_t total;
};

// chunk sums of the multi-block scans: 9 words per chunk of 4096 structures
size_t scan_parts_bytes(int64_t n) { return 8 * (3 + xrd::kPostClasses) * (size_t)((n + 4095) / 4096 + 1); }

Layout layout(int64_t n, int64_t natoms, int zmax, int64_t R, bool pg = false)
{
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o += al(bytes); return at; };
    L.geo = take(sizeof(xrd::Geo) * n);
    L.refl_cnt = take(8 * n);
    L.run_cnt = take(8 * n);
    L.refl_off = take(8 * (n + 1));
    L.tile_off = take(4 * (n + 1));
    L.order = take(4 * n);
    L.atom_bad = take(4 * n);
    L.cls_list = take(4 * xrd::kPostClasses * n);
    L.npk = take(8 * n);
    L.nfm = take(8 * n);
    L.fam_soff = take(8 * (n + 1));
    L.flags = take(kFlagBytes);
    L.coef32 = take(sizeof(xrd::Coef32) * (zmax + 1));
    L.atom32 = take(sizeof(xrd::Atom32) * natoms);
    L.atom64 = take(sizeof(xrd::Atom64) * natoms);
    L.astep = take(8 * natoms);
    L.imax = take(4 * n);
    L.cdd = take(sizeof(float4) * 4 * (zmax + 1));
    L.atomr = take(sizeof(xrd::AtomR) * natoms);
    L.tile_tab = take(8 * (R / kRunsPerTileHost + n + 1));
    L.q = take(8 * R);
    L.key = take(4 * R);
    L.runs = take(4 * R);
    L.I = take(8 * R);
    L.Eb = take(4 * R);
    L.cand_r = take(8 * (R + 1));  // also the kept-peak and family scans of the flat post passes
    L.cand_s = take(4 * (R + 1));  // also their peak starts and ids
    L.g_bkt = take(4 * (R + n));
    L.g_flag = take(R);
    L.g_pstart = take(4 * R);
    L.g_psum = take(8 * R);
    L.g_fcnt = take(4 * R);
    L.st_q = take(8 * R);
    L.st_I = take(8 * R);
    L.st_foff = take(4 * R);
    L.st_key = take(4 * R);
    L.st_mult = take(4 * R);
    L.parts = take(scan_parts_bytes(n));
    L.oparts = take(xrd::order_parts_bytes(n));
    L.pf = take(4 * (n + 1) + 8 * n + 16 + 8 * 2 * xrd::kPfScanBlocksMax + 64);
    L.pf_rec = take(16 * R);  // records of the flat post passes
    L.fkg = take(pg ? 8 * R : 0);    // family keys under the caller's point group (that mode only)
    L.pf_sfk = take(pg ? 8 * R : 0);
    L.total = o;
    return L;
}

// Workspace of the broadened-pattern / gradient path: the geometry prefix of
// the pattern layout plus the per-reflection state kept for the backward pass.
struct LayoutG {
    size_t geo, refl_cnt, run_cnt, refl_off, tile_off, order, atom_bad, tile_tab, flags, coef32, atom32, atom64,
        astep;
    size_t q, key, runs, Fx, Ig, tb, td, perm, U, V, aorder, parts, oparts;
    size_t total;
};

LayoutG layout_grad(int64_t n, int64_t natoms, int zmax, int64_t R)
{
    LayoutG L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o += al(bytes); return at; };
    L.geo = take(sizeof(xrd::Geo) * n);
    L.refl_cnt = take(8 * n);
    L.run_cnt = take(8 * n);
    L.refl_off = take(8 * (n + 1));
    L.tile_off = take(4 * (n + 1));
    L.order = take(4 * n);
    L.atom_bad = take(4 * n);
    L.flags = take(kFlagBytes);
    L.coef32 = take(sizeof(xrd::Coef32) * (zmax + 1));
    L.atom32 = take(sizeof(xrd::Atom32) * natoms);
    L.atom64 = take(sizeof(xrd::Atom64) * natoms);
    L.astep = take(8 * natoms);
    L.tile_tab = take(8 * (R / kRunsPerTileHost + n + 1));
    L.q = take(8 * R);
    L.key = take(4 * R);
    L.runs = take(4 * R);
    L.Fx = take(16 * R);
    L.Ig = take(4 * R);
    L.tb = take(4 * R);
    L.td = take(4 * R);
    L.perm = take(4 * R);
    L.U = take(4 * R);
    L.V = take(4 * R);
    L.aorder = take(4 * n);
    L.parts = take(scan_parts_bytes(n));
    L.oparts = take(xrd::order_parts_bytes(n));
    L.total = o;
    return L;
}

int64_t refl_capacity_grad(int64_t n, int64_t natoms, int zmax, size_t ws_bytes)
{
    const size_t fixed = layout_grad(n, natoms, zmax, 0).total;
    if (ws_bytes < fixed) return -1;
    int64_t lo = 0, hi = (int64_t)((ws_bytes - fixed) / 32) + 1;
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (layout_grad(n, natoms, zmax, mid).total <= ws_bytes) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Largest reflection capacity whose layout fits in ws_bytes.
int64_t refl_capacity(int64_t n, int64_t natoms, int zmax, size_t ws_bytes, bool pg = false)
{
    const size_t fixed = layout(n, natoms, zmax, 0, pg).total;
    if (ws_bytes < fixed) return -1;
    // layout(R).total grows with R: binary search for the largest R that fits
    int64_t lo = 0, hi = (int64_t)((ws_bytes - fixed) / 64) + 1;
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (layout(n, natoms, zmax, mid, pg).total <= ws_bytes) lo = mid;
        else hi = mid;
    }
    return lo;
}

int check_opts(xrd_handle* h, const xrd_opts* o)
{
    if (!o) return fail(h, XRD_EINVAL, "opts is NULL");
    if (!(o->lambda > 0.0) || !std::isfinite(o->lambda)) return fail(h, XRD_EINVAL, "lambda must be finite and > 0");
    if (!(o->tt_min >= 0.0 && o->tt_min < o->tt_max && o->tt_max <= 180.0))
        return fail(h, XRD_EINVAL, "need 0 <= tt_min < tt_max <= 180");
    if (!(o->tt_tol >= XRD_MIN_TT_TOL) || !std::isfinite(o->tt_tol))
        return fail(h, XRD_EINVAL, "tt_tol must be finite and >= 1e-9 degrees");
    if (!(o->rel_cutoff >= 0.0 && o->rel_cutoff < 1.0)) return fail(h, XRD_EINVAL, "rel_cutoff must be in [0, 1)");
    if (o->scaled != 0 && o->scaled != 1) return fail(h, XRD_EINVAL, "scaled must be 0 or 1");
    if (o->precision < XRD_FP64 || o->precision > XRD_FP32_PHASEFIX) return fail(h, XRD_EINVAL, "unknown precision");
    if (o->tile != -1 && o->tile != 64 && o->tile != 128) return fail(h, XRD_EINVAL, "tile must be -1, 64 or 128");
    if (o->reserved != 0) return fail(h, XRD_EINVAL, "reserved must be 0");
    return XRD_OK;
}

// launch shape of the structure-factor kernel for this call
void sf_shape(const xrd_handle* h, const xrd_opts* o, int& rb, int& warps, int& runs)
{
    rb = o->tile == 64 ? 2 : (o->tile == 128 ? 4 : h->sf_rb);
    warps = (o->precision == XRD_FP32_PHASEFIX) ? h->sf_warps : 2;
    runs = (o->precision == XRD_FP32_PHASEFIX && o->tile == -1 && rb == 4) ? h->sf_runs : 0;
}

int check_batch(xrd_handle* h, const xrd_batch* b)
{
    if (!b) return fail(h, XRD_EINVAL, "batch is NULL");
    if (b->n_struct < 0) return fail(h, XRD_EINVAL, "n_struct < 0");
    if (b->n_atoms < 0) return fail(h, XRD_EINVAL, "n_atoms < 0");
    if (b->zmax < 0 || b->zmax > xrd::kZmaxLimit) return fail(h, XRD_EINVAL, "zmax must be in 0..255");
    if (b->n_struct > 0 && (!b->lattice || !b->atom_off)) return fail(h, XRD_EINVAL, "lattice/atom_off is NULL");
    if (!b->coef) return fail(h, XRD_EINVAL, "coef is NULL");
    if (b->n_atoms > 0 && (!b->frac || !b->Z || !b->occ || !b->B)) return fail(h, XRD_EINVAL, "atom array is NULL");
    return XRD_OK;
}

int check_grid(xrd_handle* h, const xrd_grid* g, int& W, double& sigma)
{
    if (!g) return fail(h, XRD_EINVAL, "grid is NULL");
    if (!(g->dt > 0.0) || !std::isfinite(g->dt) || !std::isfinite(g->t0)) return fail(h, XRD_EINVAL, "grid dt/t0 invalid");
    if (!(g->fwhm > 0.0) || !std::isfinite(g->fwhm)) return fail(h, XRD_EINVAL, "grid fwhm must be > 0");
    if (g->n_pts <= 0 || g->reserved != 0) return fail(h, XRD_EINVAL, "grid n_pts must be > 0, reserved 0");
    sigma = g->fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    const double w = std::ceil(6.0 * sigma / g->dt);
    if (w > 1e6) return fail(h, XRD_EINVAL, "grid spacing too fine for the Gaussian window");
    W = (int)w;
    if (xrd::broaden_smem_bytes(g->n_pts, W) > 200 * 1024) return fail(h, XRD_EINVAL, "grid has too many points");
    return XRD_OK;
}

// sphere radii from the 2-theta range (Bragg's law), on the host in FP64
void radii(const xrd_opts* o, double& r2min, double& r2max, double& rmax)
{
    const double tmin = 2.0 * std::sin(o->tt_min * (xrd::kPi / 360.0)) / o->lambda;
    const double tmax = 2.0 * std::sin(o->tt_max * (xrd::kPi / 360.0)) / o->lambda;
    r2min = tmin * tmin;
    r2max = tmax * tmax;
    rmax = std::sqrt(r2max);
}

xrd::GeomArgs geom_args(const xrd_batch* b, const xrd_opts* o, const Layout& L, char* ws, int64_t cap_refl,
                        int64_t* totals, int32_t* status, int rb)
{
    xrd::GeomArgs g{};
    g.n_struct = b->n_struct;
    g.zmax = b->zmax;
    g.n_atoms = b->n_atoms;
    g.rb = rb;
    radii(o, g.r2min, g.r2max, g.rmax);
    g.cap_refl = cap_refl;
    g.lattice = b->lattice;
    g.atom_off = b->atom_off;
    g.frac = b->frac;
    g.Z = b->Z;
    g.occ = b->occ;
    g.B = b->B;
    g.coef = b->coef;
    g.geo = (xrd::Geo*)(ws + L.geo);
    g.coef32 = (xrd::Coef32*)(ws + L.coef32);
    g.atom32 = (xrd::Atom32*)(ws + L.atom32);
    g.atom64 = (xrd::Atom64*)(ws + L.atom64);
    g.refl_cnt = (int64_t*)(ws + L.refl_cnt);
    g.run_cnt = (int64_t*)(ws + L.run_cnt);
    g.runs = (int*)(ws + L.runs);
    g.astep = (float2*)(ws + L.astep);
    g.work = (unsigned long long*)(ws + L.flags + kWorkOffset);
    g.refl_off = (int64_t*)(ws + L.refl_off);
    g.tile_off = (int*)(ws + L.tile_off);
    g.order = (int*)(ws + L.order);
    g.atom_bad = (int*)(ws + L.atom_bad);
    g.tile_tab = (int2*)(ws + L.tile_tab);
    g.cls_list = (int*)(ws + L.cls_list);
    g.abort_flag = (int*)(ws + L.flags);
    g.enum_ctr = g.abort_flag + 26;
    g.totals = totals;
    g.status = status;
    g.q = (double*)(ws + L.q);
    g.key = (uint32_t*)(ws + L.key);
    g.parts = (long long*)(ws + L.parts);
    g.oparts = xrd::order_parts_bytes(b->n_struct) ? (int*)(ws + L.oparts) : nullptr;
    g.imax = (unsigned*)(ws + L.imax);
    g.cdd = (float4*)(ws + L.cdd);
    g.atomr = (xrd::AtomR*)(ws + L.atomr);
    return g;
}

}  // namespace

namespace xrd {
int handle_device(const xrd_handle* h) { return h ? h->device : -1; }
int set_error(xrd_handle* h, int code, const char* msg)
{
    if (h) h->err = msg;
    return code;
}
}  // namespace xrd

extern "C" {

int xrd_create(xrd_handle** h, int device)
{
    if (!h) return XRD_EINVAL;
    *h = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return XRD_ECUDA;
    if (device < 0 || device >= ndev) return XRD_EINVAL;
    xrd_handle* p = new xrd_handle();
    p->device = device;
    DeviceGuard g(device);
    e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) { xrd_destroy(p); return XRD_ECUDA; }
    for (int i = 0; i < kEvents; i++) {
        e = cudaEventCreate(&p->ev[i]);
        if (e != cudaSuccess) { xrd_destroy(p); return XRD_ECUDA; }
    }
    for (int i = 0; i < xrd::kPostStreams - 1; i++) {
        e = cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->join[i], cudaEventDisableTiming);
        if (e != cudaSuccess) { xrd_destroy(p); return XRD_ECUDA; }
    }
    e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->front, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->order_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->atoms_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&p->wbuf, 64);
    if (e != cudaSuccess) { xrd_destroy(p); return XRD_ECUDA; }
    p->ttab = xrd::init_tables(0);  // device tables (2-theta, re-evaluation), once per handle, legacy stream
    p->rtab = xrd::init_refine_tables(0);
    e = cudaStreamSynchronize(0);
    if (e != cudaSuccess || !p->ttab || !p->rtab.sc || !p->rtab.ex) { xrd_destroy(p); return XRD_ECUDA; }
    *h = p;
    return XRD_OK;
}

void xrd_destroy(xrd_handle* h)
{
    if (!h) return;
    DeviceGuard g(h->device);
    for (int i = 0; i < kEvents; i++)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    for (int i = 0; i < xrd::kPostStreams - 1; i++) {
        if (h->side[i]) cudaStreamDestroy(h->side[i]);
        if (h->join[i]) cudaEventDestroy(h->join[i]);
    }
    if (h->fork) cudaEventDestroy(h->fork);
    for (cudaEvent_t ev : {h->front, h->order_done, h->atoms_done})
        if (ev) cudaEventDestroy(ev);
    if (h->qbuf) cudaFree(h->qbuf);
    if (h->wbuf) cudaFree(h->wbuf);
    if (h->pg) cudaFree(h->pg);
    delete h;
}

const char* xrd_last_error(const xrd_handle* h) { return h ? h->err.c_str() : "NULL handle"; }

int xrd_set_refine(xrd_handle* h, int enabled)
{
    if (!h) return XRD_EINVAL;
    if (enabled != 0 && enabled != 1) return fail(h, XRD_EINVAL, "refine must be 0 or 1");
    h->refine = enabled;
    return XRD_OK;
}

int xrd_set_profiling(xrd_handle* h, int enabled)
{
    if (!h) return XRD_EINVAL;
    if (enabled < 0 || enabled > 2) return fail(h, XRD_EINVAL, "profiling mode must be 0, 1 or 2");
    h->profiling = enabled;
    return XRD_OK;
}

int xrd_stage_times(xrd_handle* h, float* ms, int n)
{
    if (!h || (!ms && n > 0)) return -XRD_EINVAL;
    if (!h->recorded) return 0;
    DeviceGuard g(h->device);
    const int m = n < kStages + 1 ? n : kStages + 1;  // the pattern stages, then the augmented profile sum
    const bool aug = h->recorded == 3, sf_only = h->recorded == 2;
    cudaError_t e = cudaEventSynchronize(h->ev[aug ? kEvents - 1 : (sf_only ? kRefineStage + 1 : kStages)]);
    if (e != cudaSuccess) return -cuda_fail(h, e, "xrd_stage_times");
    for (int i = 0; i < m; i++) {
        ms[i] = 0.f;
        if (i == kStages) {
            if (aug) e = cudaEventElapsedTime(&ms[i], h->ev[kEvents - 2], h->ev[kEvents - 1]);
        } else if (!aug && (!sf_only || i == kSfStage || i == kRefineStage)) {
            e = cudaEventElapsedTime(&ms[i], h->ev[i], h->ev[i + 1]);
        }
        if (e != cudaSuccess) return -cuda_fail(h, e, "xrd_stage_times");
    }
    return m;
}

// Friedel-unique reflection count of every structure into cnt (host), on `st` (synchronised);
// the scratch is the handle's own.
static int count_reflections(xrd_handle* h, const xrd_batch* b, const xrd_opts* o, cudaStream_t st,
                             std::vector<int64_t>& cnt)
{
    const int64_t n = b->n_struct;
    cnt.assign(n, 0);
    if (n == 0) return XRD_OK;
    const size_t need = al(sizeof(xrd::Geo) * n) + al(8 * n) + al(16);
    if (h->qbuf_bytes < need) {
        if (h->qbuf) cudaFree(h->qbuf);
        h->qbuf = nullptr;
        h->qbuf_bytes = 0;
        cudaError_t e = cudaMalloc(&h->qbuf, need);
        if (e != cudaSuccess) return cuda_fail(h, e, "xrd_query_sizes: cudaMalloc");
        h->qbuf_bytes = need;
    }
    Layout L{};
    L.geo = 0;
    L.refl_cnt = al(sizeof(xrd::Geo) * n);
    xrd::GeomArgs a{};
    a.n_struct = (int)n;
    radii(o, a.r2min, a.r2max, a.rmax);
    a.lattice = b->lattice;
    a.geo = (xrd::Geo*)((char*)h->qbuf + L.geo);
    a.refl_cnt = (int64_t*)((char*)h->qbuf + L.refl_cnt);
    a.enum_ctr = (int*)((char*)h->qbuf + L.refl_cnt + al(8 * n));  // the counting kernel's claim counter
    cudaMemsetAsync(a.enum_ctr, 0, 16, st);
    xrd::launch_count_only(a, st);
    cudaError_t e = cudaMemcpyAsync(cnt.data(), a.refl_cnt, 8 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "reflection count");
    return XRD_OK;
}

int xrd_reflection_counts(xrd_handle* h, const xrd_batch* b, const xrd_opts* o, int64_t* counts, void* stream)
{
    if (!h) return XRD_EINVAL;
    h->err.clear();
    int rc = check_batch(h, b);
    if (rc) return rc;
    if ((rc = check_opts(h, o))) return rc;
    if (!counts && b->n_struct > 0) return fail(h, XRD_EINVAL, "counts is NULL");
    DeviceGuard g(h->device);
    std::vector<int64_t> cnt;
    if ((rc = count_reflections(h, b, o, (cudaStream_t)stream, cnt))) return rc;
    for (size_t i = 0; i < cnt.size(); i++) counts[i] = cnt[i];
    return XRD_OK;
}

int xrd_query_sizes(xrd_handle* h, const xrd_batch* b, const xrd_opts* o, xrd_sizes* sizes, void* stream)
{
    if (!h) return XRD_EINVAL;
    h->err.clear();
    int rc = check_batch(h, b);
    if (rc) return rc;
    if ((rc = check_opts(h, o))) return rc;
    if (!sizes) return fail(h, XRD_EINVAL, "sizes is NULL");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = b->n_struct;
    memset(sizes, 0, sizeof(*sizes));
    if (n == 0) {
        sizes->ws_bytes = layout(0, b->n_atoms, b->zmax, 0, h->npg > 0).total;
        sizes->ws_grad_bytes = layout_grad(0, b->n_atoms, b->zmax, 0).total;
        return XRD_OK;
    }
    std::vector<int64_t> cnt;
    if ((rc = count_reflections(h, b, o, st, cnt))) return rc;
    int64_t tot = 0, mx = 0, tiles = 0;
    for (int64_t c : cnt) {
        tot += c;
        mx = c > mx ? c : mx;
        tiles += (c + 32 * h->sf_rb - 1) / (32 * h->sf_rb);
    }
    sizes->n_refl = tot;
    sizes->max_refl = mx;
    sizes->n_tiles = tiles;
    sizes->ws_bytes = layout(n, b->n_atoms, b->zmax, tot, h->npg > 0).total;
    sizes->ws_grad_bytes = layout_grad(n, b->n_atoms, b->zmax, tot).total;
    return XRD_OK;
}

int xrd_pattern_batch(xrd_handle* h, const xrd_batch* b, const xrd_opts* o, const xrd_pattern* out,
                      void* workspace, size_t ws_bytes, void* stream)
{
    if (!h) return XRD_EINVAL;
    h->err.clear();
    int rc = check_batch(h, b);
    if (rc) return rc;
    if ((rc = check_opts(h, o))) return rc;
    if (!out) return fail(h, XRD_EINVAL, "out is NULL");
    const int64_t n = b->n_struct;
    if (!out->peak_off || !out->fam_off || !out->totals || (n > 0 && !out->status))
        return fail(h, XRD_EINVAL, "an output pointer is NULL");
    if (out->cap_peaks < 0 || out->cap_fam < 0) return fail(h, XRD_EINVAL, "negative output capacity");
    if (out->cap_peaks > 0 && (!out->two_theta || !out->intensity || !out->d_hkl))
        return fail(h, XRD_EINVAL, "a peak output pointer is NULL");
    if (out->cap_fam > 0 && (!out->hkl || !out->mult)) return fail(h, XRD_EINVAL, "a family output pointer is NULL");
    if (out->refl_off) {
        if (out->cap_refl < 0) return fail(h, XRD_EINVAL, "negative reflection capacity");
        if (out->cap_refl > 0 && (!out->refl_hkl || !out->refl_tt || !out->refl_I))
            return fail(h, XRD_EINVAL, "a per-reflection output pointer is NULL");
    }
    if (!workspace || ((uintptr_t)workspace & 255)) return fail(h, XRD_EINVAL, "workspace must be 256-byte aligned");
    const bool pg = h->npg > 0;
    const int64_t cap_refl = refl_capacity(n, b->n_atoms, b->zmax, ws_bytes, pg);
    if (cap_refl < 0) return fail(h, XRD_ECAPACITY, "workspace smaller than the per-structure part");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    const Layout L = layout(n, b->n_atoms, b->zmax, cap_refl, pg);
    int rb, warps, runs;
    sf_shape(h, o, rb, warps, runs);
    xrd::GeomArgs ga = geom_args(b, o, L, ws, cap_refl, out->totals, out->status, rb);
    ga.sctab = h->rtab.sc;
    ga.runs_mode = runs;
    ga.enum_threads = h->enum_threads;
    ga.out_flags = out->flags;
    const bool refine = h->refine && o->precision != XRD_FP64;

    const int prof = h->profiling;
    unsigned rec_flags = 0;  // inside a stream capture, stage events become timed graph nodes
    if (prof) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
            rec_flags = cudaEventRecordExternal;
    }
    int stage = 0;
    auto mark = [&]() {  // mode 2 marks only the ends of the structure-factor and re-evaluation stages
        if (prof == 1 || (prof == 2 && stage >= kSfStage && stage <= kRefineStage + 1))
            cudaEventRecordWithFlags(h->ev[stage], st, rec_flags);
        stage++;
    };
    const bool pdl = prof != 1;  // programmatic launches where no stage event separates two kernels
    cudaMemsetAsync(ws + L.flags, 0, kFlagBytes, st);
    mark();
    // the input-only front beside the enumeration: order (needed by the scan), then
    // coefficients and atoms (needed by the structure factor)
    cudaStream_t side = h->side[0];
    ga.atoms_set_geo = 0;
    cudaEventRecord(h->front, st);
    cudaStreamWaitEvent(side, h->front, 0);
    xrd::launch_order(ga, side, false);
    cudaEventRecord(h->order_done, side);
    xrd::launch_coef(ga, side, true);
    xrd::launch_atoms(ga, side, true);
    cudaEventRecord(h->atoms_done, side);
    xrd::launch_prep(ga, st, false);
    mark();
    mark();  // the atom packing stage runs on the side stream: nothing on this one
    xrd::launch_count(ga, st, pdl);
    mark();
    cudaStreamWaitEvent(st, h->order_done, 0);
    xrd::launch_scan_refl(ga, st, false);
    mark();
    xrd::launch_emit(ga, st, pdl);
    mark();
    cudaStreamWaitEvent(st, h->atoms_done, 0);

    xrd::SfArgs sa{};
    sa.n_struct = (int)n;
    sa.precision = o->precision;
    sa.zmax = b->zmax;
    sa.tile = 32 * rb;
    sa.rb = rb;
    sa.warps = warps;
    sa.runs_mode = runs;
    sa.run_cnt = ga.run_cnt;
    sa.runs = ga.runs;
    sa.astep = ga.astep;
    sa.grid = h->sms;
    sa.lambda = o->lambda;
    sa.atom_off = b->atom_off;
    sa.refl_off = ga.refl_off;
    sa.tile_off = ga.tile_off;
    sa.tile_tab = ga.tile_tab;
    sa.tile_counter = ga.abort_flag + 2;
    sa.abort_flag = ga.abort_flag;
    sa.coef32 = ga.coef32;
    sa.coef = b->coef;
    sa.atom32 = ga.atom32;
    sa.atom64 = ga.atom64;
    sa.q = ga.q;
    sa.key = ga.key;
    if (o->precision == XRD_FP64) sa.I = (double*)(ws + L.I);
    else sa.If = (float*)(ws + L.I);
    sa.F = nullptr;
    if (refine) {
        sa.Eb = (float*)(ws + L.Eb);
        sa.Es = (int*)(ws + L.g_fcnt);  // free until the post-processing
        sa.eps_k = kRefineEpsK;
        sa.tau = kRefineTau;
        sa.imax = ga.imax;
    }
    xrd::launch_sf(sa, st, false);
    mark();
    if (refine) {
        xrd::RefineArgs ra{};
        ra.n_struct = (int)n;
        ra.zmax = b->zmax;
        ra.grid = h->sms;
        ra.lambda = o->lambda;
        ra.l2f = (float)(o->lambda * o->lambda * 0.25);
        ra.l2h = ra.l2f;
        ra.l2l = (float)(o->lambda * o->lambda * 0.25 - (double)ra.l2h);
        ra.tau = kRefineTau;
        ra.cref = (float)(o->rel_cutoff > 0.0 ? o->rel_cutoff : kRefineFloorNoCut);
        ra.abort_flag = ga.abort_flag;
        ra.nref = (unsigned long long*)(ws + L.flags + kRefinedOffset);
        ra.cand_r = (int64_t*)(ws + L.cand_r);
        ra.cand_s = (int*)(ws + L.cand_s);
        ra.refl_off = ga.refl_off;
        ra.atom_off = b->atom_off;
        ra.q = ga.q;
        ra.key = ga.key;
        ra.If = sa.If;
        ra.Eb = sa.Eb;
        ra.Es = sa.Es;
        ra.imax = ga.imax;
        ra.atomr = ga.atomr;
        ra.cdd = ga.cdd;
        ra.sc = h->rtab.sc;
        ra.ex = h->rtab.ex;
        ra.atom_bad = ga.atom_bad;
        xrd::launch_refine(ra, st, prof == 0);
    }
    mark();

    xrd::PostArgs pa{};
    pa.n_struct = (int)n;
    pa.geo = ga.geo;
    pa.scaled = o->scaled;
    pa.lambda = o->lambda;
    pa.tol = o->tt_tol;
    pa.cutoff = o->rel_cutoff;
    pa.r2min = ga.r2min;
    pa.r2max = ga.r2max;
    pa.l2d = o->lambda * o->lambda * 0.25;
    pa.ttab = h->ttab;
    // gaps never exceed 180 degrees: a larger tolerance merges everything
    pa.ttol = o->tt_tol > 180.0 ? INFINITY : (float)tan(o->tt_tol * (xrd::kPi / 720.0));
    pa.lo3 = (float)(ga.r2min * std::sqrt(ga.r2min));
    pa.hi3 = (float)(ga.r2max * std::sqrt(ga.r2max));
    pa.l2f = (float)pa.l2d;
    pa.lhf = (float)(o->lambda * 0.5);
    pa.refl_off = ga.refl_off;
    pa.abort_flag = ga.abort_flag;
    pa.q = ga.q;
    pa.key = ga.key;
    pa.I = sa.I;
    pa.If = sa.If;
    pa.cls_list = ga.cls_list;
    pa.cls_cnt = ga.abort_flag + xrd::kFlagClsCnt;
    pa.cls_next = ga.abort_flag + xrd::kFlagClsNext;
    pa.pf_bar = ga.abort_flag + xrd::kFlagPfBar;
    pa.pf_bar_extra = h->bar_extra;
    pa.atom_bad = ga.atom_bad;
    pa.status = out->status;
    pa.totals = out->totals;
    pa.grid = h->sms;
    pa.g_bkt = (int*)(ws + L.g_bkt);
    pa.g_flag = (uint8_t*)(ws + L.g_flag);
    pa.g_pstart = (int*)(ws + L.g_pstart);
    pa.g_psum = (double*)(ws + L.g_psum);
    pa.g_fcnt = (int*)(ws + L.g_fcnt);
    pa.st_q = (double*)(ws + L.st_q);
    pa.st_I = (double*)(ws + L.st_I);
    pa.st_foff = (int*)(ws + L.st_foff);
    pa.st_key = (uint32_t*)(ws + L.st_key);
    pa.st_mult = (int*)(ws + L.st_mult);
    pa.npk = (int64_t*)(ws + L.npk);
    pa.nfm = (int64_t*)(ws + L.nfm);
    pa.l2h = (float)pa.l2d;
    pa.l2l = (float)(pa.l2d - (double)pa.l2h);
    {
        char* pf = ws + L.pf;
        pa.pf_parts = (long long*)pf;
        pa.pf_smax = (unsigned long long*)(pf + 8 * 2 * xrd::kPfScanBlocksMax);
        pa.pf_voff = (int*)(pf + 8 * 2 * xrd::kPfScanBlocksMax + 8 * n);
        pa.pf_scal = pa.pf_voff + (n + 1);
        pa.pf_pst = (int*)(ws + L.cand_s);
        pa.pf_pj = (int*)(ws + L.Eb);
        pa.pf_kidx = (int*)(ws + L.cand_r);
        pa.pf_fidx = pa.pf_kidx + (cap_refl + 1);
        pa.pf_rec = (xrd::PfRec*)(ws + L.pf_rec);
        pa.pf_rI = (double*)(ws + L.cand_r);  // until the kept-peak scan
    }
    if (pg) {
        pa.pg = h->pg;
        pa.npg = h->npg;
        pa.fkg = (const unsigned long long*)(ws + L.fkg);
        pa.pf_sfk = (unsigned long long*)(ws + L.pf_sfk);
    }
    if (out->refl_off && out->cap_refl > 0) {
        pa.cap_refl = out->cap_refl;
        pa.refl_hkl = out->refl_hkl;
        pa.refl_tt = out->refl_tt;
        pa.refl_I = out->refl_I;
    }
    if (pg) xrd::launch_pg_keys(pa, (unsigned long long*)(ws + L.fkg), st);
    {  // the size classes run concurrently: fork to the side streams, join back
        cudaStream_t cs[xrd::kPostStreams] = {st};
        cudaEventRecord(h->fork, st);
        for (int i = 1; i < xrd::kPostStreams; i++) {
            cs[i] = h->side[i - 1];
            cudaStreamWaitEvent(cs[i], h->fork, 0);
        }
        xrd::launch_post(pa, cs);
        for (int i = 1; i < xrd::kPostStreams; i++) {
            cudaEventRecord(h->join[i - 1], cs[i]);
            cudaStreamWaitEvent(st, h->join[i - 1], 0);
        }
    }
    mark();

    xrd::CompactArgs ca{};
    ca.n_struct = (int)n;
    ca.parts = (long long*)(ws + L.parts);
    ca.grid = h->sms;
    ca.cap_peaks = out->cap_peaks;
    ca.cap_fam = out->cap_fam;
    ca.refl_off = ga.refl_off;
    ca.abort_flag = ga.abort_flag;
    ca.npk = pa.npk;
    ca.nfm = pa.nfm;
    ca.fam_soff = (int64_t*)(ws + L.fam_soff);
    ca.st_q = pa.st_q;
    ca.st_I = pa.st_I;
    ca.l2h = (float)pa.l2d;
    ca.l2l = (float)(pa.l2d - (double)ca.l2h);
    ca.ttab = h->ttab;
    ca.st_foff = pa.st_foff;
    ca.st_key = pa.st_key;
    ca.fi = pa.If != nullptr;
    ca.st_mult = pa.st_mult;
    ca.out_abort = ga.abort_flag + 1;
    ca.out = *out;
    xrd::launch_compact(ca, st);
    mark();
    h->recorded = prof;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "xrd_pattern_batch launch");
    return XRD_OK;
}

int xrd_set_point_group(xrd_handle* h, const int32_t* ops, int n_ops)
{
    if (!h) return XRD_EINVAL;
    h->err.clear();
    if (n_ops < 0 || n_ops > xrd::kMaxPgOps) return fail(h, XRD_EINVAL, "a point group has 0 to 48 operations");
    if (n_ops > 0 && !ops) return fail(h, XRD_EINVAL, "point-group operations are NULL");
    int8_t host[xrd::kMaxPgOps * 9] = {};
    for (int i = 0; i < 9 * n_ops; i++) {
        if (ops[i] < -1 || ops[i] > 1) return fail(h, XRD_EINVAL, "point-group matrix entries must be -1, 0 or 1");
        host[i] = (int8_t)ops[i];
    }
    DeviceGuard g(h->device);
    if (!h->pg) {
        cudaError_t e = cudaMalloc(&h->pg, sizeof(host));
        if (e != cudaSuccess) return cuda_fail(h, e, "xrd_set_point_group: cudaMalloc");
    }
    cudaError_t e = cudaMemcpy(h->pg, host, sizeof(host), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "xrd_set_point_group: cudaMemcpy");
    h->npg = n_ops;
    return XRD_OK;
}

int xrd_test_flat_barrier(xrd_handle* h, int extra)
{
    if (!h) return XRD_EINVAL;
    if (extra < 0 || extra > 1024) return fail(h, XRD_EINVAL, "extra must be in 0..1024");
    h->bar_extra = extra;
    return XRD_OK;
}

int xrd_set_enum_threads(xrd_handle* h, int threads)
{
    if (!h) return XRD_EINVAL;
    if (threads != 64 && threads != 128 && threads != 256 && threads != 512 && threads != 1024)
        return fail(h, XRD_EINVAL, "enumeration threads must be 64, 128, 256, 512 or 1024");
    h->enum_threads = threads;
    return XRD_OK;
}

int xrd_work_counts(xrd_handle* h, const xrd_batch* b, const void* workspace, void* stream, int64_t* counts)
{
    if (!h || !b || !workspace || !counts) return XRD_EINVAL;
    h->err.clear();
    if (b->n_struct < 0) return fail(h, XRD_EINVAL, "n_struct must be >= 0");
    DeviceGuard dg(h->device);
    // the per-structure arrays sit before every per-reflection array: any capacity gives their offsets
    const Layout L = layout(b->n_struct, b->n_atoms, b->zmax, 0);
    char* ws = (char*)const_cast<void*>(workspace);
    xrd::GeomArgs ga{};
    ga.n_struct = b->n_struct;
    ga.atom_off = b->atom_off;
    ga.refl_cnt = (int64_t*)(ws + L.refl_cnt);
    ga.run_cnt = (int64_t*)(ws + L.run_cnt);
    ga.work = (unsigned long long*)(ws + L.flags + kWorkOffset);
    uint64_t w[4] = {0, 0, 0, 0};
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(h->wbuf, 0, 64, st);
    if (e == cudaSuccess) {
        xrd::launch_work(ga, h->wbuf, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(w, h->wbuf, 3 * sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + 3, ws + L.flags + kRefinedOffset, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "xrd_work_counts");
    for (int i = 0; i < 4; i++) counts[i] = (int64_t)w[i];
    return XRD_OK;
}

int xrd_set_sf_shape(xrd_handle* h, int tile, int warps, int runs)
{
    if (!h) return XRD_EINVAL;
    if ((tile != 64 && tile != 128) || (warps != 1 && warps != 2 && warps != 4) || (runs != 0 && runs != 1) ||
        (runs && tile != 128))
        return fail(h, XRD_EINVAL, "shape must be tile 64 or 128, warps 1, 2 or 4, runs 0 or 1 (runs: tile 128)");
    h->sf_rb = tile / 32;
    h->sf_warps = warps;
    h->sf_runs = runs;
    return XRD_OK;
}

int xrd_autotune(xrd_handle* h, const xrd_batch* b, const xrd_opts* o, const xrd_pattern* out, void* workspace,
                 size_t ws_bytes, void* stream, int32_t* best_tile, int32_t* best_warps, int32_t* best_runs)
{
    if (!h) return XRD_EINVAL;
    // (reflections per lane, warps per CTA, runs)
    static const int shapes[9][3] = {{4, 2, 0}, {4, 1, 0}, {4, 4, 0}, {2, 2, 0}, {2, 1, 0},
                                     {2, 4, 0}, {4, 1, 1}, {4, 2, 1}, {4, 4, 1}};
    const bool all = o && o->precision == XRD_FP32_PHASEFIX;
    const int nshape = all ? 9 : 2;
    const int keep_rb = h->sf_rb, keep_w = h->sf_warps, keep_runs = h->sf_runs;
    const int keep_prof = h->profiling;
    xrd_opts oo = o ? *o : xrd_opts{};
    oo.tile = -1;
    float best = 1e30f;
    int brb = keep_rb, bw = keep_w, bruns = keep_runs;
    // the stage events of mode 2 end with the structure factor, so the calls' later kernels may
    // still run when xrd_stage_times returns: the stream is synchronised before every return
    auto finish = [&](int rc) {
        DeviceGuard dg(h->device);
        const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (rc == XRD_OK && e != cudaSuccess) rc = cuda_fail(h, e, "xrd_autotune");
        return rc;
    };
    h->profiling = 1;
    for (int i = 0; i < nshape; i++) {
        h->sf_rb = all ? shapes[i][0] : (i == 0 ? 4 : 2);
        h->sf_warps = all ? shapes[i][1] : 2;
        h->sf_runs = all ? shapes[i][2] : 0;
        float t = 1e30f;
        for (int rep = 0; rep < 5; rep++) {
            const int rc = xrd_pattern_batch(h, b, &oo, out, workspace, ws_bytes, stream);
            if (rc != XRD_OK) {
                h->sf_rb = keep_rb; h->sf_warps = keep_w; h->sf_runs = keep_runs; h->profiling = keep_prof;
                return finish(rc);
            }
            float ms[kStages];
            const int m = xrd_stage_times(h, ms, kStages);
            if (m < 0) {
                h->sf_rb = keep_rb; h->sf_warps = keep_w; h->sf_runs = keep_runs; h->profiling = keep_prof;
                return finish(-m);
            }
            // the stages the shape changes: count, scan, emit (runs are built there), structure factor;
            // the minimum over four calls after one warm-up
            const float sum = m >= 6 ? ms[2] + ms[3] + ms[4] + ms[5] : 1e30f;
            if (rep > 0 && sum < t) t = sum;
        }
        if (t < best) { best = t; brb = h->sf_rb; bw = h->sf_warps; bruns = h->sf_runs; }
    }
    h->sf_rb = brb;
    h->sf_warps = bw;
    h->sf_runs = bruns;
    // then the enumeration's launch shape with that shape: one warp per structure (64-256 threads
    // per CTA) for many small structures, one CTA of 512 or 1024 threads per structure for large ones
    const int keep_et = h->enum_threads;
    float best_et = 1e30f;
    int bet = keep_et;
    for (int et : {256, 128, 64, 512, 1024}) {
        h->enum_threads = et;
        float t = 1e30f;
        for (int rep = 0; rep < 5; rep++) {
            const int rc = xrd_pattern_batch(h, b, &oo, out, workspace, ws_bytes, stream);
            float ms[kStages];
            const int m = rc == XRD_OK ? xrd_stage_times(h, ms, kStages) : -rc;
            if (rc != XRD_OK || m < 0) {
                h->enum_threads = keep_et; h->profiling = keep_prof;
                return finish(rc != XRD_OK ? rc : -m);
            }
            const float sum = m >= 6 ? ms[2] + ms[3] + ms[4] : 1e30f;  // count, scan, emit
            if (rep > 0 && sum < t) t = sum;
        }
        if (t < best_et) { best_et = t; bet = et; }
    }
    h->enum_threads = bet;
    h->profiling = keep_prof;
    if (best_tile) *best_tile = 32 * brb;
    if (best_warps) *best_warps = bw;
    if (best_runs) *best_runs = bruns;
    return finish(XRD_OK);
}

struct xrd_graph_exec {
    cudaGraphExec_t exec = nullptr;
    int device = 0;
};

int xrd_graph_create(xrd_handle* h, const xrd_batch* b, const xrd_opts* o, const xrd_pattern* out, void* workspace,
                     size_t ws_bytes, void** graph)
{
    if (!h || !graph) return XRD_EINVAL;
    *graph = nullptr;
    DeviceGuard dg(h->device);
    // the eager call below runs on a private stream: work of earlier calls on the caller's
    // streams (same workspace and outputs) must be finished first
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(h, e, "xrd_graph_create: synchronise");
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(h, e, "xrd_graph_create: stream");
    // one eager call validates the arguments and settles the per-device launch caches
    int rc = xrd_pattern_batch(h, b, o, out, workspace, ws_bytes, st);
    if (rc == XRD_OK) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "xrd_graph_create: warm-up");
    }
    cudaGraph_t g = nullptr;
    if (rc == XRD_OK) {
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "xrd_graph_create: begin capture");
    }
    if (rc == XRD_OK) {
        const int rc2 = xrd_pattern_batch(h, b, o, out, workspace, ws_bytes, st);
        e = cudaStreamEndCapture(st, &g);
        if (rc2 != XRD_OK) rc = rc2;
        else if (e != cudaSuccess) rc = cuda_fail(h, e, "xrd_graph_create: end capture");
    }
    xrd_graph_exec* x = nullptr;
    if (rc == XRD_OK) {
        x = new xrd_graph_exec();
        x->device = h->device;
        e = cudaGraphInstantiate(&x->exec, g, 0);
        if (e != cudaSuccess) {
            rc = cuda_fail(h, e, "xrd_graph_create: instantiate");
            delete x;
            x = nullptr;
        }
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(st);
    *graph = x;
    return rc;
}

int xrd_graph_launch(xrd_handle* h, void* graph, void* stream)
{
    if (!h || !graph) return XRD_EINVAL;
    xrd_graph_exec* x = (xrd_graph_exec*)graph;
    DeviceGuard dg(x->device);
    const cudaError_t e = cudaGraphLaunch(x->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "xrd_graph_launch");
    return XRD_OK;
}

void xrd_graph_destroy(void* graph)
{
    if (!graph) return;
    xrd_graph_exec* x = (xrd_graph_exec*)graph;
    DeviceGuard dg(x->device);
    if (x->exec) cudaGraphExecDestroy(x->exec);
    delete x;
}

static xrd::GradArgs grad_args(xrd_handle* h, const xrd_batch* b, const xrd_grid* g, int W, double sigma,
                               const xrd_opts* o, const LayoutG& L, char* ws)
{
    xrd::GradArgs a{};
    a.n_struct = b->n_struct;
    a.n_pts = g->n_pts;
    a.W = W;
    a.n_atoms = b->n_atoms;
    a.t0 = g->t0;
    a.dt = g->dt;
    a.sigma = sigma;
    a.l2d = o->lambda * o->lambda * 0.25;
    a.l2h = (float)a.l2d;
    a.l2l = (float)(a.l2d - (double)a.l2h);
    a.ttab = h->ttab;
    a.geo = (const xrd::Geo*)(ws + L.geo);
    a.lattice = b->lattice;
    a.refl_off = (const int64_t*)(ws + L.refl_off);
    a.atom_off = b->atom_off;
    a.abort_flag = (const int*)(ws + L.flags);
    a.q = (const double*)(ws + L.q);
    a.key = (const uint32_t*)(ws + L.key);
    a.Fx = (const float4*)(ws + L.Fx);
    a.Ig = (const float*)(ws + L.Ig);
    a.tb = (int*)(ws + L.tb);
    a.td = (float*)(ws + L.td);
    a.perm = (int*)(ws + L.perm);
    a.U = (float*)(ws + L.U);
    a.V = (float*)(ws + L.V);
    a.atom32 = (const xrd::Atom32*)(ws + L.atom32);
    a.coef32 = (const xrd::Coef32*)(ws + L.coef32);
    return a;
}

// Geometry and structure factors of the broadened and augmented paths, one
// stream: grad = true keeps strided tiles and stores F, dF/ds^2 and I for the
// adjoint; grad = false runs the tuned pattern shape and stores I only.
static void launch_front(xrd_handle* h, const xrd_batch* b, const xrd_opts* o, const LayoutG& L, char* ws,
                         int64_t cap_refl, int32_t* status, int64_t* totals, cudaStream_t st, bool grad)
{
    const int64_t n = b->n_struct;
    xrd::GeomArgs ga{};
    ga.n_struct = (int)n;
    ga.zmax = b->zmax;
    ga.n_atoms = b->n_atoms;
    ga.sctab = h->rtab.sc;
    int rb, warps, runs;
    sf_shape(h, o, rb, warps, runs);
    ga.rb = rb;
    ga.runs_mode = grad ? 0 : runs;
    ga.enum_threads = grad ? 256 : h->enum_threads;
    radii(o, ga.r2min, ga.r2max, ga.rmax);
    ga.cap_refl = cap_refl;
    ga.lattice = b->lattice;
    ga.atom_off = b->atom_off;
    ga.frac = b->frac;
    ga.Z = b->Z;
    ga.occ = b->occ;
    ga.B = b->B;
    ga.coef = b->coef;
    ga.geo = (xrd::Geo*)(ws + L.geo);
    ga.coef32 = (xrd::Coef32*)(ws + L.coef32);
    ga.atom32 = (xrd::Atom32*)(ws + L.atom32);
    ga.atom64 = (xrd::Atom64*)(ws + L.atom64);
    ga.refl_cnt = (int64_t*)(ws + L.refl_cnt);
    ga.run_cnt = (int64_t*)(ws + L.run_cnt);
    ga.runs = (int*)(ws + L.runs);
    ga.astep = ga.runs_mode ? (float2*)(ws + L.astep) : nullptr;
    ga.work = (unsigned long long*)(ws + L.flags + kWorkOffset);
    ga.refl_off = (int64_t*)(ws + L.refl_off);
    ga.tile_off = (int*)(ws + L.tile_off);
    ga.order = (int*)(ws + L.order);
    ga.atom_bad = (int*)(ws + L.atom_bad);
    ga.atoms_set_geo = 1;  // atoms run before the enumeration here
    ga.tile_tab = (int2*)(ws + L.tile_tab);
    ga.abort_flag = (int*)(ws + L.flags);
    ga.enum_ctr = ga.abort_flag + 26;
    ga.totals = totals;
    ga.status = status;
    ga.q = (double*)(ws + L.q);
    ga.key = (uint32_t*)(ws + L.key);
    ga.parts = (long long*)(ws + L.parts);
    ga.oparts = xrd::order_parts_bytes(n) ? (int*)(ws + L.oparts) : nullptr;
    cudaMemsetAsync(ws + L.flags, 0, kFlagBytes, st);
    xrd::launch_prep(ga, st, false);
    xrd::launch_coef(ga, st, true);
    xrd::launch_atoms(ga, st, true);
    xrd::launch_order(ga, st, true);
    xrd::launch_count(ga, st, true);
    xrd::launch_scan_refl(ga, st, true);
    xrd::launch_emit(ga, st, true);
    xrd::SfArgs sa{};
    sa.n_struct = (int)n;
    sa.precision = XRD_FP32_PHASEFIX;
    sa.zmax = b->zmax;
    sa.tile = 32 * rb;
    sa.rb = rb;
    sa.warps = grad ? 2 : warps;
    sa.runs_mode = ga.runs_mode;
    sa.run_cnt = ga.run_cnt;
    sa.runs = ga.runs;
    sa.astep = ga.astep;
    sa.grid = h->sms;
    sa.lambda = o->lambda;
    sa.atom_off = b->atom_off;
    sa.refl_off = ga.refl_off;
    sa.tile_off = ga.tile_off;
    sa.tile_tab = ga.tile_tab;
    sa.tile_counter = ga.abort_flag + 2;
    sa.abort_flag = ga.abort_flag;
    sa.coef32 = ga.coef32;
    sa.coef = b->coef;
    sa.atom32 = ga.atom32;
    sa.atom64 = ga.atom64;
    sa.q = ga.q;
    sa.key = ga.key;
    if (grad) {
        sa.Fx = (float4*)(ws + L.Fx);
        sa.Ig = (float*)(ws + L.Ig);
    } else {
        sa.If = (float*)(ws + L.Ig);
    }
    xrd::launch_sf(sa, st, true);
}

int xrd_pattern_broadened(xrd_handle* h, const xrd_batch* b, const xrd_opts* o, const xrd_grid* grid, float* y,
                          int32_t* status, int64_t* totals, void* workspace, size_t ws_bytes, void* stream)
{
    if (!h) return XRD_EINVAL;
    h->err.clear();
    int rc = check_batch(h, b);
    if (rc) return rc;
    if ((rc = check_opts(h, o))) return rc;
    if (o->precision != XRD_FP32_PHASEFIX) return fail(h, XRD_EINVAL, "the broadened path runs XRD_FP32_PHASEFIX");
    int W;
    double sigma;
    if ((rc = check_grid(h, grid, W, sigma))) return rc;
    const int64_t n = b->n_struct;
    if (!totals || (n > 0 && (!y || !status))) return fail(h, XRD_EINVAL, "an output pointer is NULL");
    if (!workspace || ((uintptr_t)workspace & 255)) return fail(h, XRD_EINVAL, "workspace must be 256-byte aligned");
    const int64_t cap_refl = refl_capacity_grad(n, b->n_atoms, b->zmax, ws_bytes);
    if (cap_refl < 0) return fail(h, XRD_ECAPACITY, "workspace smaller than the per-structure part");
    DeviceGuard dg(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    const LayoutG L = layout_grad(n, b->n_atoms, b->zmax, cap_refl);
    launch_front(h, b, o, L, ws, cap_refl, status, totals, st, true);
    xrd::GradArgs gr = grad_args(h, b, grid, W, sigma, o, L, ws);
    gr.y = y;
    xrd::launch_broaden(gr, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "xrd_pattern_broadened launch");
    return XRD_OK;
}

int xrd_pattern_augmented(xrd_handle* h, const xrd_batch* b, const xrd_opts* o, const xrd_grid* grid,
                          const xrd_augment* aug, float* y, int32_t* status, int64_t* totals, void* workspace,
                          size_t ws_bytes, void* stream)
{
    if (!h) return XRD_EINVAL;
    h->err.clear();
    int rc = check_batch(h, b);
    if (rc) return rc;
    if ((rc = check_opts(h, o))) return rc;
    if (o->precision != XRD_FP32_PHASEFIX) return fail(h, XRD_EINVAL, "the augmented path runs XRD_FP32_PHASEFIX");
    if (!grid) return fail(h, XRD_EINVAL, "grid is NULL");
    if (!(grid->dt > 0.0) || !std::isfinite(grid->dt) || !std::isfinite(grid->t0))
        return fail(h, XRD_EINVAL, "grid dt/t0 invalid");
    if (grid->n_pts <= 0 || grid->n_pts > (1 << 22) || grid->reserved != 0)
        return fail(h, XRD_EINVAL, "grid n_pts must be in 1 .. 2^22, reserved 0");
    const double reach = std::max(std::fabs(o->tt_min - grid->t0), std::fabs(o->tt_max - grid->t0)) / grid->dt;
    if (!(reach < (double)(1 << 22))) return fail(h, XRD_EINVAL, "2-theta range more than 2^22 grid steps from t0");
    const int64_t n = b->n_struct;
    if (!aug || !totals || (n > 0 && (!y || !status))) return fail(h, XRD_EINVAL, "an output pointer is NULL");
    if (n > 0 && (!aug->fwhm || !aug->eta)) return fail(h, XRD_EINVAL, "aug fwhm and eta are required");
    if ((aug->po_dir == nullptr) != (aug->po_r == nullptr))
        return fail(h, XRD_EINVAL, "aug po_dir and po_r must be both set or both NULL");
    if ((aug->noise_z == nullptr) != (aug->noise_sigma == nullptr))
        return fail(h, XRD_EINVAL, "aug noise_z and noise_sigma must be both set or both NULL");
    const int64_t nblk = (grid->n_pts + 1023) / 1024;
    if (n * nblk > INT32_MAX) return fail(h, XRD_EINVAL, "n_struct x grid blocks exceeds the launch limit");
    if (!workspace || ((uintptr_t)workspace & 255)) return fail(h, XRD_EINVAL, "workspace must be 256-byte aligned");
    const int64_t cap_refl = refl_capacity_grad(n, b->n_atoms, b->zmax, ws_bytes);
    if (cap_refl < 0) return fail(h, XRD_ECAPACITY, "workspace smaller than the per-structure part");
    DeviceGuard dg(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    const LayoutG L = layout_grad(n, b->n_atoms, b->zmax, cap_refl);
    launch_front(h, b, o, L, ws, cap_refl, status, totals, st, false);
    xrd::AugArgs a{};
    a.n_struct = (int)n;
    a.n_pts = grid->n_pts;
    a.t0 = grid->t0;
    a.dt = grid->dt;
    a.inv_dt = 1.0 / grid->dt;
    const double l2d = o->lambda * o->lambda * 0.25;
    a.l2h = (float)l2d;
    a.l2l = (float)(l2d - (double)a.l2h);
    a.ttab = h->ttab;
    a.geo = (const xrd::Geo*)(ws + L.geo);
    a.refl_off = (const int64_t*)(ws + L.refl_off);
    a.abort_flag = (const int*)(ws + L.flags);
    a.q = (const double*)(ws + L.q);
    a.key = (const uint32_t*)(ws + L.key);
    a.Ig = (const float*)(ws + L.Ig);
    a.fwhm = aug->fwhm;
    a.eta = aug->eta;
    a.po_dir = aug->po_dir;
    a.po_r = aug->po_r;
    a.noise_z = aug->noise_z;
    a.noise_sigma = aug->noise_sigma;
    a.aorder = (int*)(ws + L.aorder);
    a.status = status;
    a.totals = totals;
    a.y = y;
    if (h->profiling) cudaEventRecord(h->ev[kEvents - 2], st);
    xrd::launch_aug(a, st);
    if (h->profiling) {
        cudaEventRecord(h->ev[kEvents - 1], st);
        h->recorded = 3;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "xrd_pattern_augmented launch");
    return XRD_OK;
}

int xrd_pattern_grad(xrd_handle* h, const xrd_batch* b, const xrd_opts* o, const xrd_grid* grid, const float* dL_dy,
                     float* d_frac, float* d_B, float* d_lattice, void* workspace, size_t ws_bytes, void* stream)
{
    if (!h) return XRD_EINVAL;
    h->err.clear();
    int rc = check_batch(h, b);
    if (rc) return rc;
    if ((rc = check_opts(h, o))) return rc;
    if (o->precision != XRD_FP32_PHASEFIX) return fail(h, XRD_EINVAL, "the broadened path runs XRD_FP32_PHASEFIX");
    int W;
    double sigma;
    if ((rc = check_grid(h, grid, W, sigma))) return rc;
    const int64_t n = b->n_struct;
    if (n > 0 && (!dL_dy || !d_lattice)) return fail(h, XRD_EINVAL, "an input/output pointer is NULL");
    if (b->n_atoms > 0 && (!d_frac || !d_B)) return fail(h, XRD_EINVAL, "an output pointer is NULL");
    if (!workspace || ((uintptr_t)workspace & 255)) return fail(h, XRD_EINVAL, "workspace must be 256-byte aligned");
    const int64_t cap_refl = refl_capacity_grad(n, b->n_atoms, b->zmax, ws_bytes);
    if (cap_refl < 0) return fail(h, XRD_ECAPACITY, "workspace smaller than the per-structure part");
    DeviceGuard dg(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    const LayoutG L = layout_grad(n, b->n_atoms, b->zmax, cap_refl);
    xrd::GradArgs gr = grad_args(h, b, grid, W, sigma, o, L, ws);
    gr.dLdy = dL_dy;
    gr.d_frac = d_frac;
    gr.d_B = d_B;
    gr.d_lat = d_lattice;
    xrd::launch_grad(gr, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "xrd_pattern_grad launch");
    return XRD_OK;
}

}  // extern "C"
