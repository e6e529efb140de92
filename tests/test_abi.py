"""Host-only checks of the C ABI: the library builds for sm_103a, loads without
a GPU, exports every entry point declared in include/cbct.h, and rejects bad
geometry descriptions before touching the device."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1001_0599_gb300 import build, cbct
    build.build()
    return cbct.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cbct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cbct_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for required in ("cbct_geometry_create", "cbct_forward_project", "cbct_back_project",
                     "cbct_tv_denoise", "cbct_reconstruct"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_library_is_built_for_sm_103a(lib):
    from paper_1001_0599_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def _desc(cbct, **kw):
    ang = np.linspace(0, 2 * math.pi, 4, endpoint=False)
    d = dict(nx=8, ny=8, nz=8, dx=1.0, dy=1.0, dz=1.0, nu=16, nv=12, du=1.0, dv=1.0, sad=100.0, sdd=150.0,
             n_views=4, step_ratio=0.5)
    d.update(kw)
    keep = np.ascontiguousarray(ang)
    desc = cbct.GeometryDesc(d["nx"], d["ny"], d["nz"], d["dx"], d["dy"], d["dz"], d["nu"], d["nv"], d["du"],
                             d["dv"], d["sad"], d["sdd"], d["n_views"],
                             keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), d["step_ratio"])
    return desc, keep


@pytest.mark.parametrize("bad", [dict(nx=0), dict(dz=0.0), dict(du=-1.0), dict(n_views=0),
                                 dict(sad=5.0), dict(sdd=104.0), dict(step_ratio=-1.0),
                                 dict(sad=float("nan"))])
def test_geometry_create_rejects_bad_descriptions(lib, bad):
    from paper_1001_0599_gb300 import cbct
    desc, keep = _desc(cbct, **bad)
    h = ctypes.c_void_p()
    st = lib.cbct_geometry_create(ctypes.byref(desc), ctypes.byref(h))
    assert st == 1  # CBCT_ERR_INVALID_ARG, reported before any device call
    assert h.value is None
    assert len(lib.cbct_last_error()) > 0


def test_null_arguments_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.cbct_geometry_create(None, ctypes.byref(h)) == 1
    assert lib.cbct_prolongate(0, 1, 1, None, None, None) == 1
    lib.cbct_geometry_destroy(None)


def test_status_codes_match_header():
    from paper_1001_0599_gb300 import cbct
    src = open(os.path.join(ROOT, "include", "cbct.h")).read()
    for code, name in cbct.STATUS.items():
        m = re.search(name + r"\s*=\s*(\d+)", src)
        assert m and int(m.group(1)) == code


def test_struct_layouts_match_header_sizes():
    # the ctypes mirrors must agree with the C structs: compile a probe
    import subprocess
    import tempfile
    from paper_1001_0599_gb300 import cbct
    code = """
#include <stdio.h>
#include "cbct.h"
int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(cbct_geometry_desc), sizeof(cbct_tv_params),
 sizeof(cbct_tv_stats), sizeof(cbct_recon_params), sizeof(cbct_iter_stats), sizeof(cbct_recon_stats),
 sizeof(cbct_server_config), sizeof(cbct_scan_result), sizeof(cbct_server_info));return 0;}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(code)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(x) for x in subprocess.check_output([exe]).split()]
    mine = [ctypes.sizeof(t) for t in (cbct.GeometryDesc, cbct.TvParams, cbct.TvStats, cbct.ReconParams,
                                       cbct.IterStats, cbct.ReconStats, cbct.ServerConfig, cbct.ScanResult,
                                       cbct.ServerInfo)]
    assert sizes == mine
