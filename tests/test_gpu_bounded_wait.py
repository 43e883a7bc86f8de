"""The bounded device-side wait of the flat post-processing passes.

The passes for structures above 6144 reflections run as one cooperative kernel
whose passes are separated by a grid-wide barrier, each wait bounded to about a
second. The test hook makes the barrier wait for an arrival that never comes (a
flag nothing sets): the call must still complete, the structures of those passes
report XRD_ETIMEOUT with no peaks, the other structures are untouched, and the
next call on the same handle gives the normal result."""
import time

import numpy as np
import pytest

from paper_2602_11709_gb300 import synth

pytestmark = pytest.mark.gpu


def _peaks(res, s):
    return [np.asarray(res[k][s]) for k in ("peak_tt", "peak_I", "peak_fam_off", "fam_hkl", "fam_mult")]


def test_flat_barrier_wait_runs_out(gpu_lib):
    xrd = gpu_lib
    bl, o = synth.large()
    bs, _ = synth.small()
    b = synth.concat([bl.subset(np.arange(2)), bs.subset(np.arange(6))])
    h = xrd.Handle(0)
    try:
        counts = h.reflection_counts(xrd.DeviceBatch.from_host(b), xrd.make_opts(o))
        flat = counts > 6144
        assert flat.sum() == 2 and (~flat).sum() == 6
        ref = xrd.compute(b, o, "fp32_phasefix", handle=h)
        assert np.all(ref["status"] == xrd.XRD_OK)
        h.test_flat_barrier(1)
        t0 = time.time()
        got = xrd.compute(b, o, "fp32_phasefix", handle=h)
        elapsed = time.time() - t0
        h.test_flat_barrier(0)
        again = xrd.compute(b, o, "fp32_phasefix", handle=h)
    finally:
        h.test_flat_barrier(0)
        h.close()
    assert elapsed < 60.0
    assert np.all(got["status"][flat] == xrd.XRD_ETIMEOUT)
    assert np.all(got["status"][~flat] == xrd.XRD_OK)
    assert int(got["totals"][3]) == 2
    for s in range(b.n_struct):
        if flat[s]:
            assert len(got["peak_tt"][s]) == 0
        else:
            for x, y in zip(_peaks(got, s), _peaks(ref, s)):
                assert np.array_equal(x, y)
    assert np.all(again["status"] == xrd.XRD_OK)
    for s in range(b.n_struct):
        for x, y in zip(_peaks(again, s), _peaks(ref, s)):
            assert np.array_equal(x, y)
