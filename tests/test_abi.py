"""The C ABI library loads and exports every entry point include/tvr.h declares
(no GPU needed: nothing here launches work)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tvr.h")


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^TVR_API\s+[\w\s\*]+?\b(tvr_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def built():
    from paper_1105_4002_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for must in ["tvr_build_system", "tvr_phi_and_grad", "tvr_project_Q", "tvr_solve_gp",
                 "tvr_solve_gpbb", "tvr_solve_upn", "tvr_system_free"]:
        assert must in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    # nothing beyond the boundary is exported
    extra = [n for n in exported if n.startswith("tvr_") and n not in declared()]
    assert not extra, extra


def test_ctypes_binding_covers_the_header(built):
    import paper_1105_4002_gb300 as pkg
    from paper_1105_4002_gb300 import _capi
    L = pkg.lib()
    assert set(_capi.SIGNATURES) == set(declared())
    for name in declared():
        assert getattr(L, name) is not None
    assert L.tvr_status_str(-4) == b"TVR_ERR_LINESEARCH"


def test_struct_layouts_match_header(built):
    """ctypes struct sizes equal the C sizes (checked with a tiny C program)."""
    import ctypes
    from paper_1105_4002_gb300 import _capi
    prog = r'''
#include <stdio.h>
#include "tvr.h"
int main(void) { printf("%zu %zu %zu\n", sizeof(tvr_geometry), sizeof(tvr_solve_opts),
                        sizeof(tvr_solve_info)); return 0; }
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert sizes == [ctypes.sizeof(_capi.Geometry), ctypes.sizeof(_capi.SolveOpts),
                     ctypes.sizeof(_capi.SolveInfo)]


def test_defaults_and_argument_errors_without_gpu(built):
    """Entry points that validate arguments before touching the device."""
    import ctypes
    import paper_1105_4002_gb300 as pkg
    from paper_1105_4002_gb300 import _capi
    L = pkg.lib()
    o = _capi.SolveOpts()
    L.tvr_solve_opts_default(ctypes.byref(o))
    assert (o.k_max, o.gpbb_K, o.gpbb_max_trials, o.bt_max) == (20000, 2, 12, 60)
    assert (o.gpbb_sigma, o.gpbb_beta0, o.rho_L, o.L_bar, o.mu_bar) == (0.1, 0.95, 2.0, 1.0, 0.1)
    h = ctypes.c_void_p()
    assert L.tvr_build_system(None, 0, None, ctypes.byref(h)) == _capi.TVR_ERR_ARG
    g = _capi.Geometry(0, 1, 1, 1, 0, 0, None)
    assert L.tvr_build_system(ctypes.byref(g), 0, None, ctypes.byref(h)) == _capi.TVR_ERR_ARG
    assert L.tvr_phi_and_grad(None, None, None, 1.0, 1.0, None, None, None, None, None) == \
        _capi.TVR_ERR_ARG
    assert L.tvr_solve_upn(None, None, 0.0, 1.0, 1.0, None, None, None, None) == _capi.TVR_ERR_ARG
    assert b"null" in L.tvr_last_error()


def test_more_validation_without_gpu(built):
    """Option defaults added to the ABI, and argument checks that run before
    any device call: unknown storage, non-finite views, a grid too large for
    int32 voxel indices, null batch and sweep arguments."""
    import ctypes
    import numpy as np
    import paper_1105_4002_gb300 as pkg
    from paper_1105_4002_gb300 import _capi
    L = pkg.lib()
    o = _capi.SolveOpts()
    L.tvr_solve_opts_default(ctypes.byref(o))
    assert (o.gpbb_points, o.sweep_lanes, o.batch, o.use_graph) == (2, 0, 32, 1)
    h = ctypes.c_void_p()
    views = np.zeros((1, 12), np.float64)
    g = _capi.Geometry(4, 1, 4, 4, _capi.TVR_CONE, 0, views.ctypes.data)
    assert L.tvr_build_system(ctypes.byref(g), 7, None, ctypes.byref(h)) == _capi.TVR_ERR_ARG
    assert b"storage" in L.tvr_last_error()
    views[0, 3] = np.nan
    assert L.tvr_build_system(ctypes.byref(g), 0, None, ctypes.byref(h)) == _capi.TVR_ERR_ARG
    assert b"non-finite" in L.tvr_last_error()
    views[0, 3] = 0.0
    big = _capi.Geometry(1291, 1, 4, 4, _capi.TVR_CONE, 0, views.ctypes.data)  # 1291^3 > 2^31
    assert L.tvr_build_system(ctypes.byref(big), 0, None, ctypes.byref(h)) == _capi.TVR_ERR_ARG
    assert b"2^31" in L.tvr_last_error()
    assert L.tvr_solve_batch(None, 0, 3, None, None, 1e-4, 1e-4, None, None, None, None) == \
        _capi.TVR_ERR_ARG
    assert L.tvr_solve_sweep(None, 3, None, None, 1, 1e-4, 1e-4, None, None, None, None) == \
        _capi.TVR_ERR_ARG
    for code in (_capi.TVR_OK, _capi.TVR_NOT_CONVERGED, _capi.TVR_ERR_ARG):
        assert L.tvr_status_str(code)
