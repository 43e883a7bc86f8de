"""Thin Python binding of the C ABI in include/xrd.h (argument marshalling only).

Device memory, streams and host<->device copies come from PyTorch; every step
of the pattern computation runs in the library's CUDA kernels. There is no CPU
fallback: if the compiled library is missing, load() raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libxrd.so")

XRD_OK, XRD_EINVAL, XRD_ECAPACITY, XRD_ECUDA, XRD_ETIMEOUT = 0, 1, 2, 3, 4
XRD_FP64, XRD_FP32_PHASE64, XRD_FP32_PHASEFIX = 0, 1, 2
XRD_MIN_TT_TOL = 1e-9  # smallest merge tolerance the library accepts, degrees
XRD_NOALLOC_SCRATCH_BYTES = 64 << 20  # fixed device scratch of xrd_pattern_batch_noalloc
PRECISIONS = {"fp64": XRD_FP64, "fp32_phase64": XRD_FP32_PHASE64, "fp32_phasefix": XRD_FP32_PHASEFIX}
STAGES = ["prep", "atoms", "count", "scan", "emit", "structure_factor", "refine", "post", "compact", "profile_sum"]
XRD_FLAG_HEXAGONAL = 1  # bit of the per-structure flag word: families by Miller-Bravais indices
# kernels xrd_pattern_batch launches per call: order, coef, atoms (a side stream), prep, count, scan, emit,
# structure factor, re-evaluation of weak reflections (selection and evaluation, FP32 variants), post
# (eight shared-memory size classes and one cooperative kernel of flat passes for the largest), output scan,
# compaction
LAUNCHES_PER_BATCH = 21


def launches_per_batch(n_struct: int, refine: bool = True, point_group: bool = False) -> int:
    """Kernels of one xrd_pattern_batch call: above two chunks of 4096 structures the
    largest-first order, the reflection scan and the output scan each take two kernels (chunk
    sums, then the chunks); the FP64 variant (or refine off) has no re-evaluation kernels; a
    caller's point group adds the family-key kernel."""
    return (LAUNCHES_PER_BATCH - (0 if refine else 2) + (3 if (n_struct + 4095) // 4096 > 2 else 0)
            + (1 if point_group else 0))


class xrd_batch(C.Structure):
    _fields_ = [("n_struct", C.c_int32), ("zmax", C.c_int32), ("n_atoms", C.c_int64), ("lattice", C.c_void_p),
                ("atom_off", C.c_void_p), ("frac", C.c_void_p), ("Z", C.c_void_p), ("occ", C.c_void_p),
                ("B", C.c_void_p), ("coef", C.c_void_p)]


class xrd_opts(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("tt_min", C.c_double), ("tt_max", C.c_double), ("tt_tol", C.c_double),
                ("rel_cutoff", C.c_double), ("scaled", C.c_int32), ("precision", C.c_int32), ("tile", C.c_int32),
                ("reserved", C.c_int32)]


class xrd_sizes(C.Structure):
    _fields_ = [("n_refl", C.c_int64), ("max_refl", C.c_int64), ("n_tiles", C.c_int64), ("ws_bytes", C.c_size_t),
                ("ws_grad_bytes", C.c_size_t)]


class xrd_grid(C.Structure):
    _fields_ = [("t0", C.c_double), ("dt", C.c_double), ("fwhm", C.c_double), ("n_pts", C.c_int32),
                ("reserved", C.c_int32)]


class xrd_augment(C.Structure):
    _fields_ = [("fwhm", C.c_void_p), ("eta", C.c_void_p), ("po_dir", C.c_void_p), ("po_r", C.c_void_p),
                ("noise_z", C.c_void_p), ("noise_sigma", C.c_void_p)]


class xrd_pattern(C.Structure):
    _fields_ = [("cap_peaks", C.c_int64), ("cap_fam", C.c_int64), ("peak_off", C.c_void_p),
                ("two_theta", C.c_void_p), ("intensity", C.c_void_p), ("d_hkl", C.c_void_p),
                ("fam_off", C.c_void_p), ("hkl", C.c_void_p), ("mult", C.c_void_p), ("status", C.c_void_p),
                ("totals", C.c_void_p), ("cap_refl", C.c_int64), ("refl_off", C.c_void_p), ("refl_hkl", C.c_void_p),
                ("refl_tt", C.c_void_p), ("refl_I", C.c_void_p), ("flags", C.c_void_p)]


EXPORTS = ["xrd_create", "xrd_destroy", "xrd_last_error", "xrd_query_sizes", "xrd_pattern_batch",
           "xrd_set_profiling", "xrd_stage_times", "xrd_pattern_batch_noalloc", "xrd_pattern_broadened",
           "xrd_pattern_grad", "xrd_autotune", "xrd_set_sf_shape", "xrd_graph_create", "xrd_graph_launch",
           "xrd_graph_destroy", "xrd_work_counts", "xrd_set_enum_threads", "xrd_pattern_augmented",
           "xrd_set_refine", "xrd_unit_rates", "xrd_reflection_counts", "xrd_set_point_group",
           "xrd_test_flat_barrier"]

_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library; raises if it was not built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing: build it with __graft_entry__.build()" % path)
    L = C.CDLL(path)
    L.xrd_create.argtypes = [C.POINTER(C.c_void_p), C.c_int]
    L.xrd_create.restype = C.c_int
    L.xrd_destroy.argtypes = [C.c_void_p]
    L.xrd_destroy.restype = None
    L.xrd_last_error.argtypes = [C.c_void_p]
    L.xrd_last_error.restype = C.c_char_p
    L.xrd_query_sizes.argtypes = [C.c_void_p, C.POINTER(xrd_batch), C.POINTER(xrd_opts), C.POINTER(xrd_sizes),
                                  C.c_void_p]
    L.xrd_query_sizes.restype = C.c_int
    L.xrd_pattern_batch.argtypes = [C.c_void_p, C.POINTER(xrd_batch), C.POINTER(xrd_opts), C.POINTER(xrd_pattern),
                                    C.c_void_p, C.c_size_t, C.c_void_p]
    L.xrd_pattern_batch.restype = C.c_int
    L.xrd_set_profiling.argtypes = [C.c_void_p, C.c_int]
    L.xrd_set_profiling.restype = C.c_int
    L.xrd_stage_times.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.c_int]
    L.xrd_stage_times.restype = C.c_int
    L.xrd_pattern_batch_noalloc.argtypes = [C.c_void_p, C.POINTER(xrd_batch), C.POINTER(xrd_opts),
                                            C.POINTER(xrd_pattern), C.c_void_p]
    L.xrd_pattern_batch_noalloc.restype = C.c_int
    L.xrd_pattern_broadened.argtypes = [C.c_void_p, C.POINTER(xrd_batch), C.POINTER(xrd_opts), C.POINTER(xrd_grid),
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
    L.xrd_pattern_broadened.restype = C.c_int
    L.xrd_pattern_grad.argtypes = [C.c_void_p, C.POINTER(xrd_batch), C.POINTER(xrd_opts), C.POINTER(xrd_grid),
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                   C.c_void_p]
    L.xrd_pattern_grad.restype = C.c_int
    L.xrd_pattern_augmented.argtypes = [C.c_void_p, C.POINTER(xrd_batch), C.POINTER(xrd_opts), C.POINTER(xrd_grid),
                                        C.POINTER(xrd_augment), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_size_t, C.c_void_p]
    L.xrd_pattern_augmented.restype = C.c_int
    L.xrd_autotune.argtypes = [C.c_void_p, C.POINTER(xrd_batch), C.POINTER(xrd_opts), C.POINTER(xrd_pattern),
                               C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32)]
    L.xrd_autotune.restype = C.c_int
    L.xrd_set_sf_shape.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
    L.xrd_work_counts.argtypes = [C.c_void_p, C.POINTER(xrd_batch), C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]
    L.xrd_work_counts.restype = C.c_int
    L.xrd_set_enum_threads.argtypes = [C.c_void_p, C.c_int]
    L.xrd_set_point_group.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
    L.xrd_set_point_group.restype = C.c_int
    L.xrd_test_flat_barrier.argtypes = [C.c_void_p, C.c_int]
    L.xrd_test_flat_barrier.restype = C.c_int
    L.xrd_set_enum_threads.restype = C.c_int
    L.xrd_set_refine.argtypes = [C.c_void_p, C.c_int]
    L.xrd_set_refine.restype = C.c_int
    L.xrd_unit_rates.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
    L.xrd_unit_rates.restype = C.c_int
    L.xrd_reflection_counts.argtypes = [C.c_void_p, C.POINTER(xrd_batch), C.POINTER(xrd_opts), C.c_void_p,
                                        C.c_void_p]
    L.xrd_reflection_counts.restype = C.c_int
    L.xrd_set_sf_shape.restype = C.c_int
    L.xrd_graph_create.argtypes = [C.c_void_p, C.POINTER(xrd_batch), C.POINTER(xrd_opts), C.POINTER(xrd_pattern),
                                   C.c_void_p, C.c_size_t, C.POINTER(C.c_void_p)]
    L.xrd_graph_create.restype = C.c_int
    L.xrd_graph_launch.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    L.xrd_graph_launch.restype = C.c_int
    L.xrd_graph_destroy.argtypes = [C.c_void_p]
    L.xrd_graph_destroy.restype = None
    _lib = L
    return L


class XrdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("xrd error %d: %s" % (code, msg))
        self.code = code


def _torch():
    import torch
    return torch


def check_tensor(name, t, dtype, shape, optional=False):
    """Argument check of the binding: a contiguous tensor of this dtype and shape (None when optional).
    Raises XrdError(XRD_EINVAL) otherwise, before any pointer reaches the library."""
    if t is None:
        if optional:
            return
        raise XrdError(XRD_EINVAL, "%s is required" % name)
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_contiguous():
        raise XrdError(XRD_EINVAL, "%s must be a contiguous %s tensor" % (name, dtype))
    if tuple(t.shape) != tuple(shape):
        raise XrdError(XRD_EINVAL, "%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def miller_bravais(hkl):
    """(h, k, l) rows -> (h, k, i = -h - k, l) rows: the 4-index form of hexagonal family representatives."""
    hkl = np.asarray(hkl)
    return np.stack([hkl[..., 0], hkl[..., 1], -hkl[..., 0] - hkl[..., 1], hkl[..., 2]], axis=-1)


def make_grid(g) -> xrd_grid:
    """C grid from any object with t0/dt/fwhm/n_pts."""
    return xrd_grid(float(g.t0), float(g.dt), float(g.fwhm), int(g.n_pts), 0)


def make_opts(o, precision="fp32_phasefix", tile=-1) -> xrd_opts:
    """C options from any object with wavelength/tt_min/tt_max/tt_tol/rel_cutoff/scaled."""
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return xrd_opts(float(o.wavelength), float(o.tt_min), float(o.tt_max), float(o.tt_tol), float(o.rel_cutoff),
                    int(o.scaled), p, int(tile), 0)


@dataclass
class DeviceBatch:
    """A batch resident in device memory (torch tensors) plus its C descriptor."""
    n_struct: int
    zmax: int
    n_atoms: int
    lattice: object
    atom_off: object
    frac: object
    Z: object
    occ: object
    B: object
    coef: object

    @staticmethod
    def from_host(b, device="cuda", pin=False):
        torch = _torch()

        def t(a, dt):
            x = torch.from_numpy(np.ascontiguousarray(a, dtype=dt))
            if pin:
                x = x.pin_memory()
            return x.to(device, non_blocking=pin)
        return DeviceBatch(int(b.lattice.shape[0]), int(b.zmax), int(b.frac.shape[0]), t(b.lattice, np.float64),
                           t(b.atom_off, np.int64), t(b.frac, np.float64), t(b.Z, np.int16), t(b.occ, np.float64),
                           t(b.B, np.float64), t(b.coef, np.float64))

    def c(self) -> xrd_batch:
        return xrd_batch(self.n_struct, self.zmax, self.n_atoms, self.lattice.data_ptr(), self.atom_off.data_ptr(),
                         self.frac.data_ptr(), self.Z.data_ptr(), self.occ.data_ptr(), self.B.data_ptr(),
                         self.coef.data_ptr())


class PatternBuffers:
    """Caller-owned output arrays of xrd_pattern_batch (torch device tensors). With refl=True the
    per-reflection list (Friedel-unique hkl, 2-theta, unmerged intensity) is written too."""

    def __init__(self, n_struct, cap, device="cuda", refl=False):
        torch = _torch()
        cap = max(int(cap), 1)
        self.n_struct = n_struct
        self.cap = cap
        self.peak_off = torch.zeros(n_struct + 1, dtype=torch.int64, device=device)
        self.two_theta = torch.zeros(cap, dtype=torch.float64, device=device)
        self.intensity = torch.zeros(cap, dtype=torch.float64, device=device)
        self.d_hkl = torch.zeros(cap, dtype=torch.float64, device=device)
        self.fam_off = torch.zeros(cap + 1, dtype=torch.int64, device=device)
        self.hkl = torch.zeros(cap, 3, dtype=torch.int32, device=device)
        self.mult = torch.zeros(cap, dtype=torch.int32, device=device)
        self.status = torch.zeros(max(n_struct, 1), dtype=torch.int32, device=device)
        self.totals = torch.zeros(4, dtype=torch.int64, device=device)
        self.flags = torch.zeros(max(n_struct, 1), dtype=torch.int32, device=device)
        self.refl = bool(refl)
        if self.refl:
            self.refl_off = torch.zeros(n_struct + 1, dtype=torch.int64, device=device)
            self.refl_hkl = torch.zeros(cap, 3, dtype=torch.int32, device=device)
            self.refl_tt = torch.zeros(cap, dtype=torch.float64, device=device)
            self.refl_I = torch.zeros(cap, dtype=torch.float64, device=device)

    def c(self) -> xrd_pattern:
        p = xrd_pattern(self.cap, self.cap, self.peak_off.data_ptr(), self.two_theta.data_ptr(),
                        self.intensity.data_ptr(), self.d_hkl.data_ptr(), self.fam_off.data_ptr(),
                        self.hkl.data_ptr(), self.mult.data_ptr(), self.status.data_ptr(), self.totals.data_ptr())
        p.flags = self.flags.data_ptr()
        if self.refl:
            p.cap_refl = self.cap
            p.refl_off = self.refl_off.data_ptr()
            p.refl_hkl = self.refl_hkl.data_ptr()
            p.refl_tt = self.refl_tt.data_ptr()
            p.refl_I = self.refl_I.data_ptr()
        return p

    def to_host(self):
        """Per-structure arrays, in the same layout as the oracle's batch results."""
        tot = self.totals.cpu().numpy()
        off = self.peak_off.cpu().numpy()
        npk, nfm = int(tot[1]), int(tot[2])
        tt = self.two_theta[:npk].cpu().numpy()
        I = self.intensity[:npk].cpu().numpy()
        d = self.d_hkl[:npk].cpu().numpy()
        fo = self.fam_off[:npk + 1].cpu().numpy()
        hkl = self.hkl[:nfm].cpu().numpy()
        mult = self.mult[:nfm].cpu().numpy()
        res = {"totals": tot, "status": self.status[:self.n_struct].cpu().numpy(),
               "flags": self.flags[:self.n_struct].cpu().numpy(), "peak_tt": [], "peak_I": [],
               "peak_d": [], "peak_fam_off": [], "fam_hkl": [], "fam_mult": []}
        if self.refl:
            ro = self.refl_off.cpu().numpy()
            nr = int(ro[-1]) if self.n_struct else 0
            rh, rt, ri = (self.refl_hkl[:nr].cpu().numpy(), self.refl_tt[:nr].cpu().numpy(),
                          self.refl_I[:nr].cpu().numpy())
            res["refl_hkl"] = [rh[ro[s]:ro[s + 1]] for s in range(self.n_struct)]
            res["refl_tt"] = [rt[ro[s]:ro[s + 1]] for s in range(self.n_struct)]
            res["refl_I"] = [ri[ro[s]:ro[s + 1]] for s in range(self.n_struct)]
        for s in range(self.n_struct):
            p0, p1 = int(off[s]), int(off[s + 1])
            f0 = int(fo[p0]) if p1 > p0 else 0
            f1 = int(fo[p1]) if p1 > p0 else 0
            res["peak_tt"].append(tt[p0:p1])
            res["peak_I"].append(I[p0:p1])
            res["peak_d"].append(d[p0:p1])
            res["peak_fam_off"].append(fo[p0:p1 + 1] - f0 if p1 > p0 else np.zeros(1, np.int64))
            res["fam_hkl"].append(hkl[f0:f1])
            res["fam_mult"].append(mult[f0:f1])
        return res


class HostPattern:
    """Pinned host mirror of a PatternBuffers, reused across calls.

    download() reads the totals first (they size the copies), then copies exactly
    the used prefix of every dense CSR output into page-locked memory with
    asynchronous copies on one stream, and returns numpy views of it.
    """

    def __init__(self, n_struct, cap):
        torch = _torch()
        cap = max(int(cap), 1)
        pin = dict(pin_memory=True)
        self.n_struct = n_struct
        self.peak_off = torch.zeros(n_struct + 1, dtype=torch.int64, **pin)
        self.two_theta = torch.zeros(cap, dtype=torch.float64, **pin)
        self.intensity = torch.zeros(cap, dtype=torch.float64, **pin)
        self.d_hkl = torch.zeros(cap, dtype=torch.float64, **pin)
        self.fam_off = torch.zeros(cap + 1, dtype=torch.int64, **pin)
        self.hkl = torch.zeros(cap, 3, dtype=torch.int32, **pin)
        self.mult = torch.zeros(cap, dtype=torch.int32, **pin)
        self.status = torch.zeros(max(n_struct, 1), dtype=torch.int32, **pin)
        self.totals = torch.zeros(4, dtype=torch.int64, **pin)
        self.bytes_last = 0

    def download(self, out: "PatternBuffers", stream=None) -> dict:
        torch = _torch()
        st = stream or torch.cuda.current_stream()
        with torch.cuda.stream(st):
            self.totals.copy_(out.totals, non_blocking=True)
            st.synchronize()
            npk, nfm = int(self.totals[1]), int(self.totals[2])
            n = self.n_struct
            pairs = [(self.peak_off, out.peak_off, n + 1), (self.status, out.status, n),
                     (self.two_theta, out.two_theta, npk), (self.intensity, out.intensity, npk),
                     (self.d_hkl, out.d_hkl, npk), (self.fam_off, out.fam_off, npk + 1),
                     (self.hkl, out.hkl, nfm), (self.mult, out.mult, nfm)]
            nbytes = self.totals.numel() * 8
            for dst, src, k in pairs:
                if k > 0:
                    dst[:k].copy_(src[:k], non_blocking=True)
                    nbytes += dst[:k].numel() * dst.element_size()
            st.synchronize()
        self.bytes_last = nbytes
        return {"totals": self.totals.numpy(), "peak_off": self.peak_off.numpy(), "status": self.status[:n].numpy(),
                "two_theta": self.two_theta[:npk].numpy(), "intensity": self.intensity[:npk].numpy(),
                "d_hkl": self.d_hkl[:npk].numpy(), "fam_off": self.fam_off[:npk + 1].numpy(),
                "hkl": self.hkl[:nfm].numpy(), "mult": self.mult[:nfm].numpy()}


class PatternPipeline:
    """Patterns of a stream of batches with the same sizes, two batches in flight.

    submit(host_arrays) copies one batch's inputs from pinned host memory to the
    device, queues xrd_pattern_batch and the copies of the result sizes, and
    returns the results of the previous submission (or None): the host waits
    only for that batch's sizes, then queues its output copies on a second
    stream, so a batch's device-to-host copy overlaps the next batch's work.
    Results are numpy views of pinned buffers, valid until the same buffer set
    is used again (two submissions later). flush() returns the last results.
    """

    def __init__(self, handle: "Handle", host_batch, opts: xrd_opts, sizes, depth: int = 2, device: int = 0):
        torch = _torch()
        dev = "cuda:%d" % device
        self.h = handle
        self.opts = opts
        self.depth = depth
        self.compute = torch.cuda.Stream(device=device)
        self.copy = torch.cuda.Stream(device=device)
        self.db = [DeviceBatch.from_host(host_batch, dev) for _ in range(depth)]
        self.out = [PatternBuffers(host_batch.n_struct, sizes.n_refl, dev) for _ in range(depth)]
        self.ws = [workspace(sizes.ws_bytes, dev) for _ in range(depth)]
        self.hp = [HostPattern(host_batch.n_struct, sizes.n_refl) for _ in range(depth)]
        self.sizes_ready = [torch.cuda.Event() for _ in range(depth)]
        self.copied = [torch.cuda.Event() for _ in range(depth)]
        self.pending = None  # buffer set whose output copies are not queued yet
        self.k = 0
        self.bytes_in = 0
        self.bytes_out = 0

    def _queue_outputs(self, j):
        torch = _torch()
        hp, out = self.hp[j], self.out[j]
        self.sizes_ready[j].synchronize()
        npk, nfm = int(hp.totals[1]), int(hp.totals[2])
        n = hp.n_struct
        with torch.cuda.stream(self.copy):
            self.copy.wait_event(self.sizes_ready[j])
            nbytes = 0
            for dst, src, m in ((hp.two_theta, out.two_theta, npk), (hp.intensity, out.intensity, npk),
                                (hp.d_hkl, out.d_hkl, npk), (hp.fam_off, out.fam_off, npk + 1),
                                (hp.hkl, out.hkl, nfm), (hp.mult, out.mult, nfm)):
                if m > 0:
                    dst[:m].copy_(src[:m], non_blocking=True)
                    nbytes += dst[:m].numel() * dst.element_size()
            self.copied[j].record(self.copy)
        self.bytes_out += nbytes + 8 * (n + 1) + 4 * n + 32
        return j, npk, nfm

    def _results(self, j, npk, nfm):
        hp = self.hp[j]
        self.copied[j].synchronize()
        n = hp.n_struct
        return {"totals": hp.totals.numpy(), "peak_off": hp.peak_off.numpy(), "status": hp.status[:n].numpy(),
                "two_theta": hp.two_theta[:npk].numpy(), "intensity": hp.intensity[:npk].numpy(),
                "d_hkl": hp.d_hkl[:npk].numpy(), "fam_off": hp.fam_off[:npk + 1].numpy(),
                "hkl": hp.hkl[:nfm].numpy(), "mult": hp.mult[:nfm].numpy()}

    def submit(self, host_arrays: dict):
        """host_arrays: pinned tensors lattice, atom_off, frac, Z, occ, B, coef of one batch."""
        torch = _torch()
        j = self.k % self.depth
        self.k += 1
        db, out, hp = self.db[j], self.out[j], self.hp[j]
        with torch.cuda.stream(self.compute):
            self.compute.wait_event(self.copied[j])  # the previous use of this buffer set is copied out
            for name, t in host_arrays.items():
                getattr(db, name).copy_(t, non_blocking=True)
                self.bytes_in += t.numel() * t.element_size()
            self.h.pattern_batch(db, self.opts, out, self.ws[j], stream=self.compute)
            hp.totals.copy_(out.totals, non_blocking=True)
            hp.peak_off.copy_(out.peak_off, non_blocking=True)
            hp.status[:hp.n_struct].copy_(out.status[:hp.n_struct], non_blocking=True)
            self.sizes_ready[j].record(self.compute)
        prev, self.pending = self.pending, j
        if prev is None:
            return None
        return self._results(*self._queue_outputs(prev))

    def flush(self):
        if self.pending is None:
            return None
        j, self.pending = self.pending, None
        return self._results(*self._queue_outputs(j))


class Handle:
    """An xrd_handle bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = C.c_void_p()
        rc = self.lib.xrd_create(C.byref(h), int(device))
        if rc != XRD_OK:
            raise XrdError(rc, "xrd_create failed")
        self.h = h

    def close(self):
        if self.h:
            self.lib.xrd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != XRD_OK:
            raise XrdError(rc, self.lib.xrd_last_error(self.h).decode())

    def query_sizes(self, db: DeviceBatch, opts: xrd_opts, stream=None) -> xrd_sizes:
        sz = xrd_sizes()
        b = db.c()
        self._check(self.lib.xrd_query_sizes(self.h, C.byref(b), C.byref(opts), C.byref(sz), _stream_ptr(stream)))
        return sz

    def reflection_counts(self, db: DeviceBatch, opts: xrd_opts, stream=None) -> np.ndarray:
        """Friedel-unique reflections of every structure (int64 numpy array)."""
        cnt = np.zeros(max(db.n_struct, 1), dtype=np.int64)
        b = db.c()
        self._check(self.lib.xrd_reflection_counts(self.h, C.byref(b), C.byref(opts),
                                                   C.c_void_p(cnt.ctypes.data), _stream_ptr(stream)))
        return cnt[:db.n_struct]

    def pattern_batch(self, db: DeviceBatch, opts: xrd_opts, out: PatternBuffers, ws, stream=None):
        b = db.c()
        o = out.c()
        self._check(self.lib.xrd_pattern_batch(self.h, C.byref(b), C.byref(opts), C.byref(o), C.c_void_p(ws.data_ptr()),
                                               C.c_size_t(ws.numel() * ws.element_size()), _stream_ptr(stream)))

    def pattern_batch_noalloc(self, db: DeviceBatch, opts: xrd_opts, out: PatternBuffers, stream=None):
        """xrd_pattern_batch on the library's fixed 64 MiB device scratch: no workspace, no allocation.

        For callers that may not allocate device memory when they need a pattern
        (a framework owns the memory pool, the host application forbids
        cudaMalloc, or an allocation's synchronisation would stall other work).
        Calls share the scratch: do not overlap them on the GPU.
        """
        b = db.c()
        o = out.c()
        self._check(self.lib.xrd_pattern_batch_noalloc(self.h, C.byref(b), C.byref(opts), C.byref(o),
                                                       _stream_ptr(stream)))

    def pattern_broadened(self, db: DeviceBatch, opts: xrd_opts, grid: xrd_grid, y, status, totals, ws, stream=None):
        """Gaussian-broadened patterns y [n_struct][n_pts] (float32); ws keeps the state for pattern_grad."""
        torch = _torch()
        check_tensor("y", y, torch.float32, (db.n_struct, int(grid.n_pts)))
        check_tensor("status", status, torch.int32, (db.n_struct,))
        check_tensor("totals", totals, torch.int64, (4,))
        b = db.c()
        self._check(self.lib.xrd_pattern_broadened(self.h, C.byref(b), C.byref(opts), C.byref(grid),
                                                   C.c_void_p(y.data_ptr()), C.c_void_p(status.data_ptr()),
                                                   C.c_void_p(totals.data_ptr()), C.c_void_p(ws.data_ptr()),
                                                   C.c_size_t(ws.numel() * ws.element_size()), _stream_ptr(stream)))

    def pattern_augmented(self, db: DeviceBatch, opts: xrd_opts, grid: xrd_grid, fwhm, eta, y, status, totals, ws,
                          po_dir=None, po_r=None, noise_z=None, noise_sigma=None, stream=None):
        """Augmented patterns y [n_struct][n_pts] (float32): per-structure pseudo-Voigt (fwhm, eta: float64
        device tensors [n_struct]), March-Dollase (po_dir [n_struct][3], po_r [n_struct]) and noise
        (noise_z float32 [n_struct][n_pts] standard normal draws, noise_sigma float64 [n_struct])."""
        torch = _torch()
        n, npts = db.n_struct, int(grid.n_pts)
        f64, f32 = torch.float64, torch.float32
        check_tensor("fwhm", fwhm, f64, (n,))
        check_tensor("eta", eta, f64, (n,))
        check_tensor("po_dir", po_dir, f64, (n, 3), optional=True)
        check_tensor("po_r", po_r, f64, (n,), optional=True)
        check_tensor("noise_z", noise_z, f32, (n, npts), optional=True)
        check_tensor("noise_sigma", noise_sigma, f64, (n,), optional=True)
        check_tensor("y", y, f32, (n, npts))
        check_tensor("status", status, torch.int32, (n,))
        check_tensor("totals", totals, torch.int64, (4,))
        b = db.c()
        ptr = lambda t: None if t is None else t.data_ptr()  # noqa: E731
        aug = xrd_augment(ptr(fwhm), ptr(eta), ptr(po_dir), ptr(po_r), ptr(noise_z), ptr(noise_sigma))
        self._check(self.lib.xrd_pattern_augmented(self.h, C.byref(b), C.byref(opts), C.byref(grid), C.byref(aug),
                                                   C.c_void_p(y.data_ptr()), C.c_void_p(status.data_ptr()),
                                                   C.c_void_p(totals.data_ptr()), C.c_void_p(ws.data_ptr()),
                                                   C.c_size_t(ws.numel() * ws.element_size()), _stream_ptr(stream)))

    def pattern_grad(self, db: DeviceBatch, opts: xrd_opts, grid: xrd_grid, dLdy, d_frac, d_B, d_lat, ws,
                     stream=None):
        """Gradients of L through the preceding pattern_broadened call on the same workspace."""
        torch = _torch()
        check_tensor("dLdy", dLdy, torch.float32, (db.n_struct, int(grid.n_pts)))
        check_tensor("d_frac", d_frac, torch.float32, (db.n_atoms, 3))
        check_tensor("d_B", d_B, torch.float32, (db.n_atoms,))
        check_tensor("d_lat", d_lat, torch.float32, (db.n_struct, 6))
        b = db.c()
        self._check(self.lib.xrd_pattern_grad(self.h, C.byref(b), C.byref(opts), C.byref(grid),
                                              C.c_void_p(dLdy.data_ptr()), C.c_void_p(d_frac.data_ptr()),
                                              C.c_void_p(d_B.data_ptr()), C.c_void_p(d_lat.data_ptr()),
                                              C.c_void_p(ws.data_ptr()), C.c_size_t(ws.numel() * ws.element_size()),
                                              _stream_ptr(stream)))

    def autotune(self, db: DeviceBatch, opts: xrd_opts, out: PatternBuffers, ws, stream=None):
        """Pick the fastest structure-factor launch shape for this batch; returns (tile, warps, runs)."""
        b, o = db.c(), out.c()
        tile, warps, runs = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(self.lib.xrd_autotune(self.h, C.byref(b), C.byref(opts), C.byref(o), C.c_void_p(ws.data_ptr()),
                                          C.c_size_t(ws.numel() * ws.element_size()), _stream_ptr(stream),
                                          C.byref(tile), C.byref(warps), C.byref(runs)))
        return tile.value, warps.value, runs.value

    def work_counts(self, db: DeviceBatch, ws, stream=None):
        """Structure-factor work of the last call on ws: (terms, phase-factor seeds, tiles, reflections
        re-evaluated in double-float)."""
        b = db.c()
        out = (C.c_int64 * 4)()
        self._check(self.lib.xrd_work_counts(self.h, C.byref(b), C.c_void_p(ws.data_ptr()), _stream_ptr(stream), out))
        return int(out[0]), int(out[1]), int(out[2]), int(out[3])

    def unit_rates(self):
        """Measured issue rates (lane operations per SM per clock) of MUFU sin, cos, ex2, FP32 FMA and
        FP64 FMA."""
        out = (C.c_double * 5)()
        self._check(self.lib.xrd_unit_rates(self.h, out))
        return {"mufu_sin": out[0], "mufu_cos": out[1], "mufu_ex2": out[2], "ffma": out[3], "dfma": out[4]}

    def set_refine(self, enabled: bool):
        """Re-evaluation of weak reflections of the FP32 variants (on by default; off is a diagnostic)."""
        self._check(self.lib.xrd_set_refine(self.h, int(bool(enabled))))

    def set_point_group(self, ops=None):
        """Families by the orbits of a point group: integer operations [n][3][3] (entries -1, 0, 1) acting
        on (h, k, l) as a column vector, n <= 48; None or [] restores permutation and sign."""
        if ops is None or len(ops) == 0:
            self._check(self.lib.xrd_set_point_group(self.h, None, 0))
            return
        arr = np.ascontiguousarray(np.asarray(ops, dtype=np.int32).reshape(-1, 3, 3))
        self._check(self.lib.xrd_set_point_group(self.h, arr.ctypes.data, int(arr.shape[0])))

    def test_flat_barrier(self, extra: int):
        """Test hook: the flat post passes' grid barrier waits for `extra` arrivals that never come,
        so that its bounded wait runs out (those structures report XRD_ETIMEOUT); 0 restores it."""
        self._check(self.lib.xrd_test_flat_barrier(self.h, int(extra)))

    def set_enum_threads(self, threads: int):
        self._check(self.lib.xrd_set_enum_threads(self.h, int(threads)))

    def set_sf_shape(self, tile: int, warps: int, runs: int = 0):
        self._check(self.lib.xrd_set_sf_shape(self.h, int(tile), int(warps), int(runs)))

    def graph(self, db: DeviceBatch, opts: xrd_opts, out: PatternBuffers, ws):
        """A CUDA graph of one pattern_batch call with these buffers."""
        return Graph(self, db, opts, out, ws)

    def set_profiling(self, mode):
        """0/False off, 1/True events between all stages, 2 events around the structure factor and the
        re-evaluation only."""
        self._check(self.lib.xrd_set_profiling(self.h, int(mode)))

    def stage_times(self):
        buf = (C.c_float * len(STAGES))()
        n = self.lib.xrd_stage_times(self.h, buf, len(STAGES))
        if n < 0:
            raise XrdError(-n, self.lib.xrd_last_error(self.h).decode())
        return {STAGES[i]: float(buf[i]) for i in range(n)}


class Graph:
    """Captured xrd_pattern_batch call (xrd_graph_create); keeps its buffers alive."""

    def __init__(self, handle: Handle, db: DeviceBatch, opts: xrd_opts, out: PatternBuffers, ws):
        self.handle, self.keep = handle, (db, opts, out, ws)
        b, o = db.c(), out.c()
        g = C.c_void_p()
        handle._check(handle.lib.xrd_graph_create(handle.h, C.byref(b), C.byref(opts), C.byref(o),
                                                  C.c_void_p(ws.data_ptr()),
                                                  C.c_size_t(ws.numel() * ws.element_size()), C.byref(g)))
        self.g = g

    def launch(self, stream=None):
        self.handle._check(self.handle.lib.xrd_graph_launch(self.handle.h, self.g, _stream_ptr(stream)))

    def close(self):
        if self.g:
            self.handle.lib.xrd_graph_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def workspace(nbytes: int, device="cuda"):
    """Device workspace (256-byte aligned: torch allocations are 512-byte aligned)."""
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def compute(batch, opts, precision="fp32_phasefix", handle: Handle = None, device: int = 0, refl=False):
    """One-shot convenience: upload a host batch, size, run and download the patterns (with refl=True
    also the per-reflection list)."""
    torch = _torch()
    h = handle or Handle(device)
    h.set_point_group(getattr(opts, "point_group", None))  # the options' point group, or none
    dev = "cuda:%d" % device
    db = DeviceBatch.from_host(batch, dev)
    o = make_opts(opts, precision)
    sz = h.query_sizes(db, o)
    out = PatternBuffers(db.n_struct, sz.n_refl, dev, refl=refl)
    ws = workspace(sz.ws_bytes, dev)
    h.pattern_batch(db, o, out, ws)
    torch.cuda.synchronize(device)
    res = out.to_host()
    res["sizes"] = {"n_refl": sz.n_refl, "max_refl": sz.max_refl, "n_tiles": sz.n_tiles, "ws_bytes": sz.ws_bytes}
    return res
