"""The allocation-free entry point xrd_pattern_batch_noalloc.

Callers that cannot allocate device memory when they need a pattern (code
under a framework-owned memory pool, plug-ins whose host forbids cudaMalloc,
loops that cannot afford an allocation's synchronisation) use this entry point:
it runs the pattern pipeline on a fixed 64 MiB device array owned by the
library. These tests compare it, through the C ABI, with xrd_pattern_batch on
a caller workspace, on two calls in a row (the second call finds the first
call's leftovers in the shared array). This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2602_11709_gb300 import synth

from parity import compare_batch

pytestmark = pytest.mark.gpu


def _host(out):
    return out.to_host()


def test_noalloc_matches_workspace_entry_point_twice(gpu_lib):
    import torch
    xrd = gpu_lib
    h = xrd.Handle(0)
    try:
        for prec in ("fp32_phasefix", "fp64"):
            for seed, n in ((2, 96), (12, 64)):
                b, o = synth.small(seed=seed, n=n)
                db = xrd.DeviceBatch.from_host(b)
                co = xrd.make_opts(o, prec)
                sz = h.query_sizes(db, co)
                ref_out = xrd.PatternBuffers(b.n_struct, sz.n_refl)
                ws = xrd.workspace(sz.ws_bytes)
                h.pattern_batch(db, co, ref_out, ws)
                torch.cuda.synchronize()
                ref = _host(ref_out)
                for call in range(2):
                    out = xrd.PatternBuffers(b.n_struct, sz.n_refl)
                    h.pattern_batch_noalloc(db, co, out)
                    torch.cuda.synchronize()
                    got = _host(out)
                    assert np.all(got["status"] == 0), (prec, call)
                    assert np.array_equal(got["totals"], ref["totals"]), (prec, call)
                    compare_batch(got, {**ref, "status": ref["status"]}, prec, o.rel_cutoff, o.scaled)
    finally:
        h.close()


def test_noalloc_capacity_limits(gpu_lib):
    import torch
    xrd = gpu_lib
    h = xrd.Handle(0)
    try:
        # reflections beyond the fixed scratch (1.03 million of about 105 bytes each), outputs with
        # room for every peak and family: the scratch alone is too small, flagged on the device for
        # every structure, and totals[0] gives the reflection count it would need
        b, o = synth.small()
        db = xrd.DeviceBatch.from_host(b)
        co = xrd.make_opts(o, "fp32_phasefix")
        sz = h.query_sizes(db, co)
        assert sz.ws_bytes > xrd.XRD_NOALLOC_SCRATCH_BYTES
        out = xrd.PatternBuffers(b.n_struct, sz.n_refl)
        h.pattern_batch_noalloc(db, co, out)
        torch.cuda.synchronize()
        assert np.all(out.status.cpu().numpy() == xrd.XRD_ECAPACITY)
        assert int(out.totals[3]) == b.n_struct
        assert int(out.totals[0]) == sz.n_refl
        # per-structure arrays beyond the scratch: rejected on the host before any launch
        big = xrd.xrd_batch(2_000_000, db.zmax, db.n_atoms, db.lattice.data_ptr(), db.atom_off.data_ptr(),
                            db.frac.data_ptr(), db.Z.data_ptr(), db.occ.data_ptr(), db.B.data_ptr(),
                            db.coef.data_ptr())
        po = out.c()
        rc = h.lib.xrd_pattern_batch_noalloc(h.h, C.byref(big), C.byref(co), C.byref(po), None)
        assert rc == xrd.XRD_ECAPACITY
        assert b"64 MiB" in h.lib.xrd_last_error(h.h)
        # a later normal call still works on the same scratch
        small, o2 = synth.small(n=8)
        ds = xrd.DeviceBatch.from_host(small)
        out2 = xrd.PatternBuffers(small.n_struct, 20000)
        h.pattern_batch_noalloc(ds, xrd.make_opts(o2, "fp32_phasefix"), out2)
        torch.cuda.synchronize()
        assert np.all(out2.status.cpu().numpy() == 0)
    finally:
        h.close()


def test_noalloc_after_handle_recreated(gpu_lib):
    """The scratch address is looked up per context: a handle destroyed and created again on the
    same device (same context) keeps giving the workspace entry point's results."""
    import torch
    xrd = gpu_lib
    b, o = synth.small(seed=21, n=48)
    db = xrd.DeviceBatch.from_host(b)
    co = xrd.make_opts(o, "fp32_phasefix")
    results = []
    for _ in range(2):
        h = xrd.Handle(0)
        try:
            sz = h.query_sizes(db, co)
            out = xrd.PatternBuffers(b.n_struct, sz.n_refl)
            h.pattern_batch_noalloc(db, co, out)
            ref_out = xrd.PatternBuffers(b.n_struct, sz.n_refl)
            h.pattern_batch(db, co, ref_out, xrd.workspace(sz.ws_bytes))
            torch.cuda.synchronize()
            got, ref = out.to_host(), ref_out.to_host()
            compare_batch(got, ref, "fp32_phasefix", o.rel_cutoff, o.scaled)
            results.append(got)
        finally:
            h.close()
    for s in range(b.n_struct):
        assert np.array_equal(results[0]["peak_I"][s], results[1]["peak_I"][s])
