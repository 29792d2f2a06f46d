"""The C-ABI library builds, loads and exports every entry point include/*.h declares;
host-only calls (parameter checks, workspace sizing, messages) work without a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(mpfc\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1208_2643_gb300 import mpfc
    return mpfc.load()


def test_headers_declare_entry_points():
    names = declared_functions()
    for must in ("mpfc_create", "mpfc_step", "mpfc_energy", "mpfc_mass", "mpfc_destroy", "mpfc_workspace_bytes"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params_and_workspace(lib):
    from paper_1208_2643_gb300 import mpfc
    p = mpfc.default_params()
    assert (p.m, p.n, p.nu1, p.nu2, p.coarsest) == (64, 64, 2, 2, 4)
    assert p.omega == 0.8 and p.tol == 1e-10
    b64 = mpfc.workspace_bytes(p)
    assert b64 > 0
    p2 = mpfc.default_params(m=1024, n=1024)
    b1k = mpfc.workspace_bytes(p2)
    # the level hierarchy adds a geometric 1/3 on top of the finest level's planes
    assert 1024 * 1024 * 8 * 10 < b1k < 1024 * 1024 * 8 * 20


@pytest.mark.parametrize("kw", [dict(m=63), dict(m=62), dict(h=0.0), dict(dt=-1.0), dict(omega=1.5),
                                dict(nu1=0, nu2=0), dict(precision=7), dict(guess=9), dict(max_cycles=0),
                                dict(coarsest=1),
                                dict(m=2, n=2),                 # below the 4-cell minimum per side
                                dict(m=65536, n=65536),         # more than 2^30 cells
                                dict(m=65536, n=32768),         # 2^31 cells: past the 32-bit index range
                                dict(m=16384, n=65536),         # 2^30 cells but more rows than a grid's y extent
                                dict(m=254, n=254),             # coarsening stops at 127^2 > 64 cells
                                dict(epsilon=1.5), dict(inner_cycles=65), dict(bc=5), dict(model=3),
                                dict(pinning=2),
                                dict(pinning=1, guess=2),       # learned guess: periodic, unpinned only
                                dict(bc=1, guess=2)])
def test_invalid_params_rejected(lib, kw):
    from paper_1208_2643_gb300 import mpfc
    assert mpfc.workspace_bytes(mpfc.default_params(**kw)) == 0


@pytest.mark.parametrize("m,n", [(4, 4), (4, 6), (6, 6), (8, 12), (32768, 32768), (65536, 16384)])
def test_smallest_and_largest_grids_accepted(lib, m, n):
    """A single-level grid (the coarsest solve alone) and grids up to 2^30 cells (the kernels
    index cells in 32-bit ints, and cell index plus grid stride must stay below 2^31)."""
    from paper_1208_2643_gb300 import mpfc
    b = mpfc.workspace_bytes(mpfc.default_params(m=m, n=n))
    assert b >= m * n * 8 * 10


def test_create_rejects_without_workspace(lib):
    from paper_1208_2643_gb300 import mpfc
    p = mpfc.default_params()
    h = ctypes.c_void_p()
    assert lib.mpfc_create(ctypes.byref(p), None, 0, None, ctypes.byref(h)) == mpfc.MPFC_ERR_WORKSPACE
    assert lib.mpfc_create(None, None, 0, None, ctypes.byref(h)) == mpfc.MPFC_ERR_INVALID


def test_strerror(lib):
    from paper_1208_2643_gb300 import mpfc
    for code in (0, -1, -2, -3, -4, -5):
        assert len(mpfc.strerror(code)) >= 2
