"""The C-ABI library builds, loads without a GPU, and exports every entry point that
include/snap.h declares; the Python binding names the same set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "snap.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(snap_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1901_02955_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary_calls():
    names = declared()
    for n in ["snap_init_grid", "snap_set_state", "snap_step", "snap_get_state",
              "snap_step_adjoint", "snap_free", "snap_last_error"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1901_02955_gb300 import EXPORTS
    assert sorted(EXPORTS) == declared()


def test_status_strings_without_gpu(lib):
    lib.snap_status_string.restype = ctypes.c_char_p
    assert lib.snap_status_string(0) == b"ok"
    assert b"invalid" in lib.snap_status_string(-1)


def test_invalid_descriptor_rejected_on_host(lib):
    """Validation happens before any CUDA call, so it runs without a GPU."""
    import numpy as np
    import workloads as W
    from paper_1901_02955_gb300 import capi
    w = W.warm_bubble(n=8)
    d, keep = capi.desc_from_workload(w)
    d.nx = 2
    L = capi.load()
    p = ctypes.c_void_p()
    assert L.snap_init_grid(ctypes.byref(p), ctypes.byref(d), 1) == capi.EINVAL
    assert b"nx" in L.snap_last_error(None)
    d, keep = capi.desc_from_workload(w)
    pf = np.array(w.p_bar_face)
    pf[3] *= 1.01
    d.p_bar_face = pf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.snap_init_grid(ctypes.byref(p), ctypes.byref(d), 1) == capi.EINVAL
    assert b"hydrostatic" in L.snap_last_error(None)
    d, keep = capi.desc_from_workload(w)
    d.bc[4] = capi.PERIODIC
    assert L.snap_init_grid(ctypes.byref(p), ctypes.byref(d), 1) == capi.EINVAL


def test_descriptor_layout_matches_the_header(tmp_path):
    """The ctypes mirrors of snap_grid_desc and snap_species have the C layout: a small C
    program compiled against include/snap.h prints the size and field offsets."""
    import shutil
    import subprocess
    from paper_1901_02955_gb300 import capi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    fields = [f for f, _ in capi.GridDesc._fields_]
    prog = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "snap.h"', "int main(void) {",
             '  printf("%zu %zu\\n", sizeof(snap_grid_desc), sizeof(snap_species));']
    for f in fields:
        lines.append(f'  printf("%zu\\n", offsetof(snap_grid_desc, {f}));')
    lines.append("  return 0;\n}\n")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(prog),
                           "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split()
    assert int(out[0]) == ctypes.sizeof(capi.GridDesc)
    assert int(out[1]) == ctypes.sizeof(capi.Species)
    for f, off in zip(fields, out[2:]):
        assert int(off) == getattr(capi.GridDesc, f).offset, f


def test_noslip_and_bottom_temperature_are_validated(lib):
    import workloads as W
    from paper_1901_02955_gb300 import capi
    L = capi.load()
    p = ctypes.c_void_p()
    w = W.warm_bubble(n=8)
    d, keep = capi.desc_from_workload(w)
    d.bc[4] = capi.PERIODIC
    d.bc[5] = capi.PERIODIC
    assert L.snap_init_grid(ctypes.byref(p), ctypes.byref(d), 1) == capi.EINVAL
    assert b"walls" in L.snap_last_error(None)
    d, keep = capi.desc_from_workload(w)
    d.bc[0] = 7
    assert L.snap_init_grid(ctypes.byref(p), ctypes.byref(d), 1) == capi.EINVAL
    d, keep = capi.desc_from_workload(w)
    d.T_bottom = -1.0
    assert L.snap_init_grid(ctypes.byref(p), ctypes.byref(d), 1) == capi.EINVAL
    assert b"T_bottom" in L.snap_last_error(None)


def test_empty_and_degenerate_grids_rejected_on_host(lib):
    """No domain, a NULL descriptor, an empty axis or one shorter than the three cells a
    WENO5 stencil reaches each way: SNAP_EINVAL before any CUDA call."""
    import workloads as W
    from paper_1901_02955_gb300 import capi
    L = capi.load()
    p = ctypes.c_void_p()
    w = W.warm_bubble(n=8)
    d, keep = capi.desc_from_workload(w)
    assert L.snap_init_grid(ctypes.byref(p), ctypes.byref(d), 0) == capi.EINVAL
    assert L.snap_init_grid(ctypes.byref(p), None, 1) == capi.EINVAL
    for field, value in (("nx", 0), ("nz", 0), ("nz", 2), ("ny", 0)):
        d, keep = capi.desc_from_workload(w)
        setattr(d, field, value)
        assert L.snap_init_grid(ctypes.byref(p), ctypes.byref(d), 1) == capi.EINVAL, (field, value)
