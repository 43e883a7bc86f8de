"""Host-side checks of the C ABI: the library builds, loads without a GPU, exports
every entry point declared in include/xrd.h, and the ctypes mirrors of the C
structs have the C layout."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_2602_11709_gb300 import build as pkg_build
from paper_2602_11709_gb300 import xrd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "xrd.h")


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return xrd.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(xrd_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_entry_point(lib):
    names = declared_functions()
    assert {"xrd_create", "xrd_destroy", "xrd_last_error", "xrd_query_sizes", "xrd_pattern_batch"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    assert set(xrd.EXPORTS) <= set(names)


def test_struct_layouts_match_c():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "xrd.h"
#define F(T, m) printf("%s.%s %zu\n", #T, #m, offsetof(T, m))
int main(void) {
  printf("xrd_batch %zu\nxrd_opts %zu\nxrd_sizes %zu\nxrd_pattern %zu\n", sizeof(xrd_batch), sizeof(xrd_opts),
         sizeof(xrd_sizes), sizeof(xrd_pattern));
  F(xrd_batch, n_atoms); F(xrd_batch, coef); F(xrd_opts, scaled); F(xrd_opts, reserved);
  F(xrd_sizes, ws_bytes); F(xrd_pattern, fam_off); F(xrd_pattern, totals);
  printf("xrd_augment %zu\n", sizeof(xrd_augment)); F(xrd_augment, po_r); F(xrd_augment, noise_sigma);
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    assert int(got["xrd_batch"]) == C.sizeof(xrd.xrd_batch)
    assert int(got["xrd_opts"]) == C.sizeof(xrd.xrd_opts)
    assert int(got["xrd_sizes"]) == C.sizeof(xrd.xrd_sizes)
    assert int(got["xrd_pattern"]) == C.sizeof(xrd.xrd_pattern)
    assert int(got["xrd_batch.n_atoms"]) == xrd.xrd_batch.n_atoms.offset
    assert int(got["xrd_batch.coef"]) == xrd.xrd_batch.coef.offset
    assert int(got["xrd_opts.scaled"]) == xrd.xrd_opts.scaled.offset
    assert int(got["xrd_opts.reserved"]) == xrd.xrd_opts.reserved.offset
    assert int(got["xrd_sizes.ws_bytes"]) == xrd.xrd_sizes.ws_bytes.offset
    assert int(got["xrd_pattern.fam_off"]) == xrd.xrd_pattern.fam_off.offset
    assert int(got["xrd_pattern.totals"]) == xrd.xrd_pattern.totals.offset
    assert int(got["xrd_augment"]) == C.sizeof(xrd.xrd_augment)
    assert int(got["xrd_augment.po_r"]) == xrd.xrd_augment.po_r.offset
    assert int(got["xrd_augment.noise_sigma"]) == xrd.xrd_augment.noise_sigma.offset


def test_every_struct_field_matches_c():
    """Size and every field offset of each ctypes mirror against the C compiler's layout of xrd.h."""
    structs = [xrd.xrd_batch, xrd.xrd_opts, xrd.xrd_sizes, xrd.xrd_grid, xrd.xrd_augment, xrd.xrd_pattern]
    lines = []
    for S in structs:
        lines.append('printf("%%s %%zu\\n", "%s", sizeof(%s));' % (S.__name__, S.__name__))
        for f, _ in S._fields_:
            cname = f.rstrip("_")  # lambda is a Python keyword
            lines.append('printf("%%s %%zu\\n", "%s.%s", offsetof(%s, %s));' % (S.__name__, f, S.__name__, cname))
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"xrd.h\"\nint main(void) {\n" + "\n".join(lines) + \
        "\nreturn 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    for S in structs:
        assert int(got[S.__name__]) == C.sizeof(S), S.__name__
        for f, _ in S._fields_:
            assert int(got["%s.%s" % (S.__name__, f)]) == getattr(S, f).offset, (S.__name__, f)


def test_header_constants_match_binding():
    """Return codes, precisions and the smallest merge tolerance: the #defines of xrd.h equal the
    binding's constants."""
    text = open(HEADER).read()
    m = re.search(r"#define\s+XRD_MIN_TT_TOL\s+([0-9.eE+-]+)", text)
    assert m and float(m.group(1)) == xrd.XRD_MIN_TT_TOL
    for name in ("XRD_OK", "XRD_EINVAL", "XRD_ECAPACITY", "XRD_ECUDA", "XRD_ETIMEOUT", "XRD_FP64",
                 "XRD_FP32_PHASE64", "XRD_FP32_PHASEFIX", "XRD_FLAG_HEXAGONAL"):
        m = re.search(r"#define\s+%s\s+(\d+)\b" % name, text)
        assert m and int(m.group(1)) == getattr(xrd, name), name


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = lib.xrd_create(C.byref(h), 0)
    assert rc in (xrd.XRD_ECUDA, xrd.XRD_EINVAL) and not h.value
    assert lib.xrd_last_error(None) == b"NULL handle"


def test_null_handle_arguments(lib):
    assert lib.xrd_query_sizes(None, None, None, None, None) == xrd.XRD_EINVAL
    assert lib.xrd_pattern_batch(None, None, None, None, None, 0, None) == xrd.XRD_EINVAL
    assert lib.xrd_set_profiling(None, 1) == xrd.XRD_EINVAL
    assert lib.xrd_set_refine(None, 1) == xrd.XRD_EINVAL
    assert lib.xrd_set_point_group(None, None, 0) == xrd.XRD_EINVAL
    assert lib.xrd_test_flat_barrier(None, 0) == xrd.XRD_EINVAL
    lib.xrd_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    saved = xrd._lib
    try:
        xrd._lib = None
        with pytest.raises(RuntimeError):
            xrd.load(str(tmp_path / "nope.so"))
    finally:
        xrd._lib = saved


def test_launch_count_per_call():
    """Kernels per xrd_pattern_batch call: 21 with the two re-evaluation kernels of the FP32 variants
    (19 without), three more above two chunks of 4096 structures (two-kernel order and scans), one
    more with a caller's point group (family keys)."""
    assert xrd.launches_per_batch(1024) == 21 and xrd.launches_per_batch(8192) == 21
    assert xrd.launches_per_batch(8193) == 24 and xrd.launches_per_batch(100_000) == 24
    assert xrd.launches_per_batch(1024, refine=False) == 19 and xrd.launches_per_batch(8193, refine=False) == 22
    assert xrd.launches_per_batch(1024, point_group=True) == 22


def test_binding_argument_checks():
    """The binding refuses a tensor of the wrong dtype, layout or shape before calling the library."""
    import torch
    xrd.check_tensor("y", torch.zeros(2, 5, dtype=torch.float32), torch.float32, (2, 5))
    xrd.check_tensor("po_dir", None, torch.float64, (2, 3), optional=True)
    bad = [(None, torch.float64, (2,), False),                                   # required
           (torch.zeros(2, dtype=torch.float32), torch.float64, (2,), False),    # dtype
           (torch.zeros(2, 3, dtype=torch.float64).t(), torch.float64, (3, 2), False),  # not contiguous
           (torch.zeros(3, dtype=torch.float64), torch.float64, (2,), False)]    # shape
    for t, dt, shape, opt in bad:
        with pytest.raises(xrd.XrdError):
            xrd.check_tensor("x", t, dt, shape, optional=opt)
