"""The C-ABI library builds, loads and exports every declared symbol; host-side
argument checks reject bad calls before any device work (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("defined", "sizeof"):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_17314_b300 import build, _capi
    build.build()
    return _capi.load()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib):
    from paper_2607_17314_b300 import _capi
    assert set(declared_functions()) == set(_capi.SIGNATURES)


def test_struct_layout_matches_header():
    """Field offsets of the ctypes mirrors follow the C layout rules."""
    from paper_2607_17314_b300 import _capi as C
    assert ctypes.sizeof(C.IsdfOptions) == 32 and C.IsdfOptions.stage_ms.offset == 24
    assert C.IsdfJastrow.d.offset == 16
    assert C.IsdfJastrow.nuc_xyz.offset == 24
    assert ctypes.sizeof(C.IsdfBasis) == 8 + 4 * 8


def test_workspace_queries(lib):
    assert lib.isdf_points_workspace(1000, 10) >= 8 * (2 * 1000 + 2 * 10 * 1000)
    assert lib.tc_kernel_build_workspace(100000, 2000, 0, 100000, 1) > 2 * 2048 * 100000 * 2
    assert lib.tc_kernel_build_workspace(4800, 96, 0, 4800, 0) > 0


def test_argument_errors_need_no_gpu(lib):
    from paper_2607_17314_b300 import _capi as C
    J = C.IsdfJastrow()
    J.n_types, J.d = 1, 1.0
    J.d = -1.0  # invalid
    st = lib.tc_kernel_build(None, None, None, None, 10, 2, 0, 10, ctypes.byref(J), None,
                             None, None, None, 0, None)
    assert st == C.ISDF_E_ARG
    assert b"d must be positive" in lib.isdf_last_error()
    J.d = 1.0
    st = lib.tc_kernel_build(None, None, None, None, 10, 2, 0, 10, ctypes.byref(J), None,
                             None, None, None, 0, None)
    assert st == C.ISDF_E_ARG  # null pointers
    st = lib.isdf_points(None, None, None, 10, 2, 4, 7, None, None, None, 0, None)
    assert st == C.ISDF_E_ARG


def test_product_path_has_no_oracle_import():
    """The package never imports the oracle or the input generator."""
    for f in glob.glob(os.path.join(ROOT, "paper_2607_17314_b300", "**", "*.py"), recursive=True):
        src = open(f).read()
        assert not re.search(r"^\s*(from|import)\s+(oracle|synth)\b", src, flags=re.M), f
