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


def test_struct_layout_matches_header(tmp_path):
    """Sizes and field offsets of the ctypes mirrors equal the C compiler's for
    the header's structs (a C program built against include/isdftc.h prints them)."""
    import subprocess
    from paper_2607_17314_b300 import _capi as C
    mirrors = {"isdf_options": C.IsdfOptions, "isdf_jastrow": C.IsdfJastrow,
               "isdf_basis": C.IsdfBasis}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "isdftc.h"', "int main(void) {"]
    for cname, cls in mirrors.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f[0], cname, f[0]))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            cname, field, val = line.split()
            got[(cname, field)] = int(val)
    for cname, cls in mirrors.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f in cls._fields_:
            assert got[(cname, f[0])] == getattr(cls, f[0]).offset, (cname, f[0])


def test_workspace_queries(lib):
    assert lib.isdf_points_workspace(1000, 10) >= 8 * (2 * 1000 + 2 * 10 * 1000)
    assert lib.tc_kernel_build_workspace(100000, 2000, 0, 100000, 1, None) > 2 * 2048 * 100000 * 2
    assert lib.tc_kernel_build_workspace(4800, 96, 0, 4800, 0, None) > 0


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
    fake = ctypes.c_void_p(256)
    n = C.INT(0)
    for ranks in ((0, 0), (-1, 4), (4, -1)):
        st = lib.isdf_points_fixed_rank(fake, fake, fake, 64, 4, *ranks, fake, ctypes.byref(n),
                                        fake, 1 << 30, None)
        assert st == C.ISDF_E_ARG, ranks


def test_correlator_parameters_checked_before_launch(lib):
    """Scale parameters b_I > 0 (Eq. bh-scaled) and finite d, positions and
    coefficients are required before any device work; b is not used, and not
    checked, when the correlator has no free terms."""
    from paper_2607_17314_b300 import _capi as C
    fake = ctypes.c_void_p(256)

    def build(J):
        return lib.tc_kernel_build(fake, fake, fake, fake, 64, 4, 0, 64, ctypes.byref(J), None,
                                   fake, fake, fake, 0, None)

    J = C.IsdfJastrow()
    J.n_nuc, J.n_types, J.d, J.cusp = 1, 1, 1.0, 1
    J.b[0] = 0.0                       # radial correlator: b unused
    assert build(J) == C.ISDF_E_ARG    # the zero-byte workspace fails later
    assert b"b must be positive" not in lib.isdf_last_error()
    J.n_terms = 1
    J.mno[0][0], J.mno[0][1], J.mno[0][2] = 1, 0, 0
    J.coef[0][0] = 0.1
    for b in (0.0, -1.0, float("inf"), float("nan")):
        J.b[0] = b
        assert build(J) == C.ISDF_E_ARG
        assert b"b must be positive" in lib.isdf_last_error()
    J.b[0] = 1.0
    J.coef[0][0] = float("nan")
    assert build(J) == C.ISDF_E_ARG
    assert b"coefficient not finite" in lib.isdf_last_error()
    J.coef[0][0] = 0.1
    J.nuc_xyz[0][2] = float("inf")
    assert build(J) == C.ISDF_E_ARG
    assert b"position not finite" in lib.isdf_last_error()
    J.nuc_xyz[0][2] = 0.0
    J.d = float("inf")
    assert build(J) == C.ISDF_E_ARG
    assert b"d must be positive" in lib.isdf_last_error()


def test_xtc_sizes_checked_before_launch(lib):
    """No occupied orbitals, n_occ > n_orb or an X width beyond n_orb are
    argument errors, reported before any device work."""
    from paper_2607_17314_b300 import _capi as C
    fake = ctypes.c_void_p(256)
    for n_occ, n_orb_x in ((0, 4), (9, 4), (2, 9)):
        st = lib.xtc_density_contract(fake, 8, n_occ, fake, fake, fake, 64, 16, fake, fake,
                                      n_orb_x, 0, fake, 1 << 30, None)
        assert st == C.ISDF_E_ARG, (n_occ, n_orb_x)
    st = lib.isdf_gather_pivots(fake, None, 64, 0, fake, 4, fake, None, None)
    assert st == C.ISDF_E_ARG


def test_multicentre_tensor_core_form_needs_no_gpu(lib):
    """The multi-centre tensor-core generator sizes its tables from the
    correlator and rejects term sets outside its polynomial form before any
    device work."""
    from paper_2607_17314_b300 import _capi as C
    J = C.IsdfJastrow()
    J.n_nuc, J.n_types, J.d, J.cusp = 12, 2, 1.0, 1
    for I in range(12):
        J.nuc_type[I] = I % 2
        J.nuc_xyz[I][0] = float(I)
    J.b[0] = J.b[1] = 1.0
    radial_ws = lib.tc_kernel_build_workspace(4096, 128, 0, 4096, 1, ctypes.byref(J))
    terms = [(0, 0, 2), (1, 0, 0), (1, 1, 0), (1, 1, 2), (2, 2, 2)]
    J.n_terms = len(terms)
    for k, t in enumerate(terms):
        J.mno[k][0], J.mno[k][1], J.mno[k][2] = t
        J.coef[0][k] = J.coef[1][k] = 0.01
    bh_ws = lib.tc_kernel_build_workspace(4096, 128, 0, 4096, 1, ctypes.byref(J))
    # (point, nucleus) slots: 3 gradient + 2 + 2 x 3 polynomial = 11 -> 3 float4,
    # plus f(g) and the A table
    assert bh_ws - radial_ws >= 4096 * (12 * 3 * 16 + 16 + 12 * 4)
    fake = ctypes.c_void_p(256)
    J.mno[1][0] = 4
    st = lib.tc_kernel_build(fake, fake, fake, fake, 4096, 128, 0, 4096, ctypes.byref(J), None,
                             fake, fake, fake, 1 << 30, None)
    assert st == C.ISDF_E_ARG
    assert b"tensor-core generator" in lib.isdf_last_error()
    J.mno[1][0] = 1
    for k, t in enumerate([(1, 1, 2), (1, 1, 3), (1, 1, 4)]):
        J.mno[k][0], J.mno[k][1], J.mno[k][2] = t
    st = lib.tc_kernel_build(fake, fake, fake, fake, 4096, 128, 0, 4096, ctypes.byref(J), None,
                             fake, fake, fake, 1 << 30, None)
    assert st == C.ISDF_E_ARG
    assert b"two E exponents" in lib.isdf_last_error()


def test_product_path_has_no_oracle_import():
    """The package never imports the oracle or the input generator."""
    for f in glob.glob(os.path.join(ROOT, "paper_2607_17314_b300", "**", "*.py"), recursive=True):
        src = open(f).read()
        assert not re.search(r"^\s*(from|import)\s+(oracle|synth)\b", src, flags=re.M), f


def test_undersized_workspace_rejected_before_launch(lib):
    """Every call that takes a workspace rejects one that is too small with
    ISDF_E_ARG and a message naming the bytes needed, before any device work."""
    from paper_2607_17314_b300 import _capi as C
    f = ctypes.c_void_p(256)
    n = C.INT(0)
    eps = ctypes.c_double(0.0)
    basis = C.IsdfBasis(4, 3, f, f, f, f)
    J = C.IsdfJastrow()
    J.n_types, J.d, J.cusp, J.b[0] = 1, 1.0, 1, 1.0
    opt64 = C.IsdfOptions(C.ISDF_PREC_FP64, 0, 0, 1, 0, None, 0.0, 0.0, 0, 0)
    calls = {
        "isdf_eval_orbitals": lambda: lib.isdf_eval_orbitals(ctypes.byref(basis), f, 4, f, 64, f,
                                                             f, f, 16, None),
        "isdf_points": lambda: lib.isdf_points(f, f, f, 64, 4, 8, 0, f, ctypes.byref(n), f, 16,
                                               None),
        "isdf_points_fixed_rank": lambda: lib.isdf_points_fixed_rank(
            f, f, f, 64, 4, 4, 4, f, ctypes.byref(n), f, 16, None),
        "isdf_fit": lambda: lib.isdf_fit(f, f, 64, 4, f, 8, f, f, None, None, f, 16, None),
        "tc_kernel_build": lambda: lib.tc_kernel_build(f, f, f, f, 64, 8, 0, 64, ctypes.byref(J),
                                                       None, f, f, f, 16, None),
        "tc_kernel_build (fp64)": lambda: lib.tc_kernel_build(
            f, f, f, f, 64, 8, 0, 64, ctypes.byref(J), ctypes.byref(opt64), f, f, f, 16, None),
        "tc_kernel_build_streamed": lambda: lib.tc_kernel_build_streamed(
            f, f, f, f, 64, 8, 64, 64, ctypes.byref(J), None, f, f, 16, None),
        "tc_kernel_adjoint": lambda: lib.tc_kernel_adjoint(f, f, f, f, 64, 8, ctypes.byref(J), f,
                                                           C.PRECISIONS["fp64"], f, f, 16, None),
        "xtc_density_contract": lambda: lib.xtc_density_contract(f, 4, 2, f, f, f, 64, 8, f, f, 4,
                                                                 0, f, 16, None),
        "tc_energies": lambda: lib.tc_energies(f, f, f, f, f, 8, 4, 2, f, f, 16, None),
        "isdf_points_restricted": lambda: lib.isdf_points_restricted(f, f, f, 64, 4, f, 32, 8, f,
                                                                     ctypes.byref(n), f, 16, None),
        "isdf_fit_error": lambda: lib.isdf_fit_error(f, f, 64, 4, f, 8, ctypes.byref(eps), f, 16,
                                                     None),
    }
    for name, call in calls.items():
        st = call()
        assert st == C.ISDF_E_ARG, (name, st, lib.isdf_last_error())
        assert b"workspace too small" in lib.isdf_last_error(), (name, lib.isdf_last_error())


def test_streamed_build_argument_checks(lib):
    """The streamed W build rejects the FP64 precision and ket batches that are
    not multiples of 32 before any device work, and its workspace query is 0
    for them."""
    from paper_2607_17314_b300 import _capi as C
    f = ctypes.c_void_p(256)
    J = C.IsdfJastrow()
    J.n_types, J.d, J.cusp, J.b[0] = 1, 1.0, 1, 1.0
    opt64 = C.IsdfOptions(C.ISDF_PREC_FP64, 0, 0, 1, 0, None, 0.0, 0.0, 0, 0)
    st = lib.tc_kernel_build_streamed(f, f, f, f, 4096, 64, 1024, 1024, ctypes.byref(J),
                                      ctypes.byref(opt64), f, f, 1 << 30, None)
    assert st == C.ISDF_E_ARG and b"tensor-core precisions" in lib.isdf_last_error()
    st = lib.tc_kernel_build_streamed(f, f, f, f, 4096, 64, 1024, 1000, ctypes.byref(J), None, f,
                                      f, 1 << 30, None)
    assert st == C.ISDF_E_ARG and b"multiple of 32" in lib.isdf_last_error()
    assert lib.tc_kernel_build_streamed_workspace(4096, 64, 1024, 1024, C.ISDF_PREC_FP64, None) == 0
    small = lib.tc_kernel_build_streamed_workspace(100000, 2000, 8192, 8192, 1, ctypes.byref(J))
    big = lib.tc_kernel_build_workspace(100000, 2000, 0, 100000, 1, ctypes.byref(J))
    assert 0 < small < big


def test_vmc_argument_checks(lib):
    """The VMC entry points (Sec. II.C) reject bad sizes, steps and undersized
    workspaces before any device work."""
    from paper_2607_17314_b300 import _capi as C
    fake = ctypes.c_void_p(256)
    B = C.IsdfBasis(8, 3, fake, fake, fake, fake)
    J = C.IsdfJastrow()
    J.n_nuc, J.n_types, J.n_terms, J.d, J.cusp = 2, 1, 1, 1.0, 1
    J.b[0], J.coef[0][0] = 1.0, 0.1
    J.mno[0][0] = 1
    assert lib.isdf_vmc_n_params(ctypes.byref(J)) == 3
    Z = (ctypes.c_double * 2)(1.0, 1.0)
    zp = ctypes.cast(Z, ctypes.c_void_p)
    need = lib.isdf_vmc_local_energy_workspace(8, 2, 16, ctypes.byref(J))
    assert need >= 8 * (5 * 8 * 64 + 5 * 2 * 64)

    def eloc(n_occ, ws_bytes, h=1e-5, dE=fake):
        return lib.isdf_vmc_local_energy(ctypes.byref(B), fake, 8, n_occ, fake, 16,
                                         ctypes.byref(J), zp, None, h, fake, dE, fake, ws_bytes,
                                         None)
    for n_occ in (0, 9, 65):
        assert eloc(n_occ, need) == C.ISDF_E_ARG
    assert eloc(2, need - 1) == C.ISDF_E_ARG
    assert b"workspace too small" in lib.isdf_last_error()
    assert eloc(2, need, h=0.0) == C.ISDF_E_ARG
    assert b"fd_step" in lib.isdf_last_error()
    acc = ctypes.c_void_p(512)
    for sigma, n_occ in ((0.0, 2), (float("nan"), 2), (0.5, 0)):
        st = lib.isdf_vmc_sample(ctypes.byref(B), fake, 8, n_occ, fake, 16, fake, fake, 2, sigma,
                                 acc, None)
        assert st == C.ISDF_E_ARG
    st = lib.isdf_vmc_sample(ctypes.byref(B), fake, 8, 2, fake, 16, None, None, 2, 0.5, acc, None)
    assert st == C.ISDF_E_ARG and b"random inputs" in lib.isdf_last_error()
    gw = lib.isdf_vmc_gn_step_workspace(100, 3)
    assert gw >= 8 * (3 * 100 + 100 + 3 + 9)
    assert lib.isdf_vmc_gn_step(fake, fake, 1, 3, 0.0, 1.0, None, fake, fake, fake, gw,
                                None) == C.ISDF_E_ARG
    assert lib.isdf_vmc_gn_step(fake, fake, 100, 3, -1.0, 1.0, None, fake, fake, fake, gw,
                                None) == C.ISDF_E_ARG
    assert lib.isdf_vmc_gn_step(fake, fake, 100, 3, 0.0, 1.0, None, fake, fake, fake, gw - 1,
                                None) == C.ISDF_E_ARG


def test_emulated_products_argument_checks(lib):
    """isdf_dgemm_emulated, the mode workspaces and isdf_vmc_polyak reject bad
    arguments before any device work."""
    from paper_2607_17314_b300 import _capi as C
    fake = ctypes.c_void_p(256)
    ws = lib.isdf_dgemm_emulated_workspace(300, 200, 128)
    # 8 digit planes of both operands (BF16) at the padded sizes
    assert ws >= 16 * (384 * 128 + 256 * 128)
    assert lib.isdf_dgemm_emulated(0, 5, 5, None, 5, None, 5, 1.0, 0.0, None, 5, None, 0,
                                   None) == C.ISDF_OK  # empty product: nothing to do
    for beta in (0.5, -1.0):
        assert lib.isdf_dgemm_emulated(4, 4, 4, fake, 4, fake, 4, 1.0, beta, fake, 4, fake, ws,
                                       None) == C.ISDF_E_ARG
    assert lib.isdf_dgemm_emulated(4, 4, 4, fake, 4, fake, 4, float("nan"), 0.0, fake, 4, fake,
                                   ws, None) == C.ISDF_E_ARG
    assert lib.isdf_dgemm_emulated(4, 4, 8, fake, 4, fake, 4, 1.0, 0.0, fake, 4, fake, ws,
                                   None) == C.ISDF_E_ARG  # lda < K
    assert lib.isdf_dgemm_emulated(4, 4, 4, fake, 4, fake, 4, 1.0, 0.0, fake, 4, fake, 16,
                                   None) == C.ISDF_E_ARG  # workspace too small
    assert b"workspace too small" in lib.isdf_last_error()
    assert lib.isdf_fit_workspace_mode(1000, 40, 100, 2) == 0
    assert lib.isdf_fit_workspace_mode(1000, 40, 100, 1) > lib.isdf_fit_workspace_mode(1000, 40,
                                                                                        100, 0)
    assert lib.isdf_fit_workspace_mode(1000, 40, 100, 0) == lib.isdf_fit_workspace(1000, 40, 100)
    assert lib.isdf_eval_orbitals_workspace_mode(50, 1000, 40, 3) == 0
    assert lib.isdf_eval_orbitals_workspace_mode(50, 1000, 40, 0) == \
        lib.isdf_eval_orbitals_workspace(50, 1000)
    opt = C.IsdfOptions()
    opt.fit_mode = 2
    st = lib.isdf_fit(fake, fake, 100, 4, fake, 8, fake, fake, None, ctypes.byref(opt), fake,
                      1 << 30, None)
    assert st == C.ISDF_E_ARG and b"fit_mode" in lib.isdf_last_error()
    assert lib.isdf_vmc_polyak(fake, fake, 0, 1, None) == C.ISDF_E_ARG
    assert lib.isdf_vmc_polyak(fake, fake, 4, 0, None) == C.ISDF_E_ARG
    assert lib.isdf_vmc_objective(fake, 1, fake, None) == C.ISDF_E_ARG


def test_vmc_schedule_rejects_bad_window():
    """The averaging window must lie within the refinement steps (checked on
    the host before any device work)."""
    from paper_2607_17314_b300 import api
    for n_refine, window in ((5, 0), (5, 6), (0, 1)):
        with pytest.raises(ValueError):
            api.vmc_schedule(None, None, 1, None, None, None, None, n_warm=1, n_refine=n_refine,
                             window=window, sweeps=1, sigma=0.5)


def test_binding_rejects_mismatched_shapes():
    """The Python binding passes sizes taken from one tensor together with the
    pointers of the others, so every other tensor is checked against those
    sizes on the host before anything reaches the library (a smaller tensor
    would be read or written out of bounds on the device).  CPU tensors reach
    the shape check, which comes before the device check."""
    import torch
    from paper_2607_17314_b300 import api, _capi as C
    d = torch.float64

    def z(*shape, dtype=d):
        return torch.zeros(shape, dtype=dtype)

    J = C.IsdfJastrow()
    J.n_nuc, J.n_types, J.n_terms, J.d = 2, 1, 0, 1.0
    basis = (z(4, 3), z(4, 3, dtype=torch.int32), z(4, 2), z(4, 2))
    cases = {
        "dphi": lambda: api.isdf_points(z(3, 10), z(3, 3, 9), z(10), 4),
        "w": lambda: api.isdf_points_fixed_rank(z(3, 10), z(3, 3, 10), z(9), 2, 2),
        "pivots": lambda: api.isdf_fit(z(3, 10), z(3, 3, 10), z(2, 2, dtype=torch.int32)),
        "B": lambda: api.isdf_dgemm_emulated(z(4, 5), z(6, 3)),
        "out": lambda: api.isdf_dgemm_emulated(z(4, 5), z(5, 3), out=z(3, 4)),
        "xi_grad": lambda: api.KernelBuilder(z(10, 3), z(10), z(4, 10), z(3, 4, 9), J),
        "grid_xyz": lambda: api.tc_kernel_build(z(10, 2), z(10), z(4, 10), z(3, 4, 10), J),
        "xig_host": lambda: api.tc_kernel_build_streamed(z(10, 3), z(10), z(4, 10), z(4, 4, 10), J),
        "calG": lambda: api.xtc_density_contract(z(4, 3), 1, z(4, 10), z(10), z(4, 4, 9), 1),
        "phi_piv": lambda: api.xtc_density_contract(z(5, 3), 1, z(4, 10), z(10), z(4, 4, 10), 1),
        "W": lambda: api.tc_energies(z(4, 5, 5), z(4, 4), z(3, 4), z(4, 3), z(3, 4, 3), 2),
        "needs at least 3": lambda: api.tc_energies(z(4, 4, 4), z(4, 4), z(2, 4), z(4, 3),
                                                    z(3, 4, 3), 2),
        "full X": lambda: api.tc_two_body_panel(z(4, 4, 4), z(4, 4), z(3, 4), z(4, 3), z(3, 4, 3),
                                                0, 3),
        "dphi_piv": lambda: api.tc_xtc_one_body(z(4, 4, 4), z(4, 4), z(6, 4), z(4, 3), z(3, 3, 4),
                                                1),
        "Wbar": lambda: api.tc_kernel_adjoint(z(10, 3), z(10), z(4, 10), z(3, 4, 10), J,
                                              z(4, 4, 3)),
        "mo_coef": lambda: api.isdf_eval_orbitals(*basis[:1], basis[1], basis[2], basis[3],
                                                  z(5, 2), z(10, 3)),
        "coefs": lambda: api.isdf_vmc_sample((z(4, 3), basis[1], z(4, 2), z(4, 3)), z(4, 2), 1,
                                             z(8, 2, 3), z(2, 2, 8, 3), z(2, 2, 8), 0.5),
        "walkers": lambda: api.isdf_vmc_local_energy(basis, z(4, 2), 2, z(8, 2, 3), J, [1.0, 1.0]),
        "charges": lambda: api.isdf_vmc_local_energy(basis, z(4, 2), 1, z(8, 2, 3), J, [1.0]),
        "normals": lambda: api.isdf_vmc_sample(basis, z(4, 2), 1, z(8, 2, 3), z(2, 2, 8, 2),
                                               z(2, 2, 8), 0.5),
        "uniforms": lambda: api.isdf_vmc_sample(basis, z(4, 2), 1, z(8, 2, 3), z(2, 2, 8, 3),
                                                z(2, 2, 7), 0.5),
        "dE": lambda: api.isdf_vmc_gn_step(z(8), z(3, 9), 0.0, 1.0),
        "theta": lambda: api.isdf_vmc_gn_step(z(8), z(3, 8), 0.0, 1.0, theta=z(4)),
    }
    from paper_2607_17314_b300 import proposer as PR
    P = PR.n_params()
    f32 = torch.float32
    cases.update({
        r"grid_xyz has shape \(10, 4\)": lambda: PR.features(z(3, 10), z(3, 3, 10), z(10), z(10, 4),
                                                             [[0, 0, 0]]),
        "params": lambda: PR.forward(z(P - 1, dtype=f32), z(5, 8, dtype=f32)),
        "feat": lambda: PR.forward(z(P, dtype=f32), z(5, 7, dtype=f32)),
        "labels": lambda: PR.backward(z(P, dtype=f32), z(5, 8, dtype=f32), z(4, dtype=f32), 1.0,
                                      5, z(P, dtype=f32), z(1)),
        "loss": lambda: PR.backward(z(P, dtype=f32), z(5, 8, dtype=f32), z(5, dtype=f32), 1.0,
                                    5, z(P, dtype=f32), z(2)),
        "m has shape": lambda: PR.adam(z(P, dtype=f32), z(P, dtype=f32), z(3, dtype=f32),
                                       z(P, dtype=f32), 1, 1e-3),
        "cand": lambda: PR.points_restricted(z(3, 10), z(3, 3, 10), z(10),
                                             z(2, 2, dtype=torch.int32), 2),
        "w has shape": lambda: PR.fit_error(z(3, 10), z(11), z(2, dtype=torch.int32)),
    })
    for name, call in cases.items():
        with pytest.raises(ValueError, match=name):
            call()
