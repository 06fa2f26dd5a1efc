"""The C ABI library loads and exports every entry point include/pmg.h declares, and the
host-side validation rejects bad descriptors without touching a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

import paper_2411_14977_gb300.pmg as pmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(pmg_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = pmg.load(build_if_missing=True)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_library_exports_nothing_undeclared():
    """Every exported pmg_* function is declared in include/ (no stray C-ABI entry points)."""
    import shutil
    import subprocess
    if shutil.which("nm") is None:
        pytest.skip("nm not available")
    pmg.load(build_if_missing=True)
    out = subprocess.run(["nm", "-D", "--defined-only", pmg.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = {f[2] for f in (ln.split() for ln in out.splitlines()) if len(f) == 3 and f[1] == "T"
                and f[2].startswith("pmg_")}
    assert exported == declared_functions(), (sorted(exported - declared_functions()),
                                              sorted(declared_functions() - exported))


def test_binding_covers_declared_symbols():
    assert declared_functions() <= set(pmg._SIGNATURES)


def test_default_opts():
    o = pmg.default_opts()
    assert (o.precision, o.outer, o.overlap, o.nu, o.omega, o.tol) == (0, 0, 1, 2, 0.8, 1e-10)


@pytest.mark.parametrize("mesh,opts,needle", [
    (dict(order=0), {}, "order"),
    (dict(order=11), {}, "order"),
    (dict(order=1), {}, "order must be >= 2"),
    (dict(cells_x=0), {}, "cells"),
    (dict(x1=-1.0), {}, "x1 > x0"),
    (dict(h=0.0), {}, "h > 0"),
    (dict(periodic_x=1, cells_x=6), {}, "power of two"),
    (dict(), dict(nu=0), "options"),
    (dict(), dict(overlap=2), "options"),
    (dict(), dict(precision=7), "precision"),
    (dict(), dict(outer=3), "refinement needs a mixed precision"),
    (dict(), dict(precision=2), "outer = PMG_IR"),
    (dict(), dict(precision=2, outer=1), "outer = PMG_IR"),
    (dict(), dict(fuse_residual=2), "options"),
    (dict(), dict(df64_outer=3), "options"),
    (dict(), dict(flat_kernel=4), "options"),
    (dict(), dict(flat_kernel=1032), "options"),    # bulk-staged with 32 threads
    (dict(), dict(flat_kernel=1080), "options"),    # not whole warps
    (dict(), dict(flat_kernel=1544), "options"),
    (dict(), dict(flat_kernel=13216), "options"),   # 32 x 16 = 512 threads
    (dict(), dict(flat_kernel=10404), "options"),   # 4 element columns
    (dict(), dict(flat_kernel=11603), "options"),   # 3 element rows
    (dict(), dict(flat_kernel=20808), "options"),
    (dict(), dict(flat_kernel=-2), "options"),
    (dict(), dict(outer=5), "outer"),
    (dict(), dict(outer=4, gmres_restart=0), "gmres_restart"),
    (dict(), dict(outer=4, gmres_restart=61), "gmres_restart"),
    (dict(), dict(nlevels=4, levels=[4, 2, 2, 1]), "decrease"),
    (dict(), dict(nlevels=2, levels=[4, 2]), "order to 1"),
])
def test_create_rejects_bad_input(mesh, opts, needle):
    lib = pmg.load()
    m = pmg.MeshDesc(0.0, 1.0, 1.0, 4, 2, 4, 0)
    for k, v in mesh.items():
        setattr(m, k, v)
    o = pmg.default_opts()
    for k, v in opts.items():
        if k == "levels":
            for i, p in enumerate(v):
                o.level_orders[i] = p
        else:
            setattr(o, k, v)
    h = ctypes.c_void_p()
    st = lib.pmg_create(ctypes.byref(m), ctypes.byref(o), ctypes.byref(h))
    assert st == pmg.PMG_ERR_INVALID
    assert h.value is None
    assert needle in lib.pmg_last_error().decode()


def test_null_arguments():
    lib = pmg.load()
    assert lib.pmg_create(None, None, None) == pmg.PMG_ERR_INVALID
    h = ctypes.c_void_p()
    assert lib.pmg_create(None, None, ctypes.byref(h)) == pmg.PMG_ERR_INVALID
    assert lib.pmg_destroy(None) == pmg.PMG_OK
    assert lib.pmg_solve(None, None, None, None, None, None, None) == pmg.PMG_ERR_INVALID


@pytest.mark.parametrize("code", [2, 10804, 10808, 11604, 11608, 13204, 13208, 3, 1064, 1256, 1512])
def test_tiled_level_operator_shapes_pass_validation(code):
    """Every documented tiled shape (pmg_opts.flat_kernel = 2 or 10000 + 100 EXT + ZT) and
    bulk-staged shape (3 or 1000 + threads) passes the option check; creation then stops
    only where it needs a device."""
    lib = pmg.load()
    m = pmg.MeshDesc(0.0, 1.0, 1.0, 4, 2, 4, 0)
    o = pmg.default_opts()
    o.flat_kernel = code
    h = ctypes.c_void_p()
    st = lib.pmg_create(ctypes.byref(m), ctypes.byref(o), ctypes.byref(h))
    if st != pmg.PMG_OK:
        assert "options" not in lib.pmg_last_error().decode()
    else:
        lib.pmg_destroy(h)
