"""The allocation-free energies entry point (for callers that cannot allocate
device memory, e.g. inside another framework's memory pool or on paths that
must not block on an allocator) matches the workspace entry point, call after
call, through the C ABI."""
import ctypes

import numpy as np
import pytest
import torch

from synth import workloads as wl
from oracle import orbitals, pivots, fit, wbuild, xtc

pytestmark = pytest.mark.gpu


def _case():
    w = wl.h6_chain()
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    res = pivots.select(phi, dphi, w.grid_w, w.n_mu)
    xi, xit, _ = fit.fit(phi, dphi, res.pivots)
    W, calG = wbuild.build(w.grid_xyz, w.grid_w, xi, xit, w.jastrow)
    phiP = xtc.pivot_factors(phi, res.pivots)
    dphiP = np.stack([dphi[c][:, res.pivots].T for c in range(3)])
    _, _, D = xtc.d_kernels(w.grid_w, xi, calG, xtc.g_nu(phiP, w.n_occ))
    Xp = xtc.pack_upper(xtc.x_projector(w.grid_w, xi, calG, phiP, w.n_occ))
    return w, W, D, Xp, phiP, dphiP


def test_noalloc_energies_match_workspace_call_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_17314_b300 import build
    build.build()
    from paper_2607_17314_b300 import _capi as C
    lib = C.load()
    w, W, D, Xp, phiP, dphiP = _case()
    dev = [torch.as_tensor(np.ascontiguousarray(a)).cuda() for a in (W, D, Xp, phiP, dphiP)]
    ptr = [ctypes.c_void_p(t.data_ptr()) for t in dev]
    n_mu, n_orb = phiP.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ref = (ctypes.c_double * 3)()
    ws = torch.empty(lib.tc_energies_workspace(n_mu, w.n_occ), dtype=torch.uint8, device="cuda")
    C.check("tc_energies", lib.tc_energies(*ptr, n_mu, n_orb, w.n_occ, ref,
                                           ctypes.c_void_p(ws.data_ptr()), ws.numel(), stream))
    for _ in range(2):
        out = (ctypes.c_double * 3)()
        C.check("tc_energies_noalloc",
                lib.tc_energies_noalloc(*ptr, n_mu, n_orb, w.n_occ, out, stream))
        for a, b in zip(out, ref):
            assert abs(a - b) <= 1e-10 * abs(b) + 1e-14, (list(out), list(ref))
    # beyond the fixed scratch the call is rejected with a clear error
    st = lib.tc_energies_noalloc(*ptr, 4096, n_orb, 24, out, stream)
    assert st == C.ISDF_E_ARG
    assert b"allocation-free call" in lib.isdf_last_error()
