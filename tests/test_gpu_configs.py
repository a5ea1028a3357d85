"""Parity at the full sizes of the H50-chain and benzene workloads (the
bench's workload and the largest one), on what the oracle can compute there.

H50 chain (100,000 points, 550 functions -> 400 orbitals, N_mu = 2000):
  - orbitals and gradients on the GPU against the oracle at 4096 sampled
    points (1e-12 relative);
  - the fused pivot selection bit-exact against the oracle on the GPU's own
    orbitals (identical inputs), truncated to 500 points for host time;
  - the fit at the full N_mu = 2000: backward error of the normal equations
    on 256 sampled grid columns (1e-10) and forward agreement with the oracle's
    Cholesky solve of those columns within the Gram's condition number.
Benzene (271,800 points, 1200 orbitals): orbitals at sampled points and the
fused pivots bit-exact, truncated to 200 points.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

from synth import workloads as wl
from oracle import orbitals, pivots, fit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_17314_b300 import build
    build.build()
    from paper_2607_17314_b300 import api
    return api


def _cu(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dt).cuda()


def _orbitals(api, w, mode=0):
    b = w.basis
    return api.isdf_eval_orbitals(_cu(b.center), _cu(b.powers, torch.int32), _cu(b.exps),
                                  _cu(b.coefs), _cu(w.mo_coef), _cu(w.grid_xyz), mode=mode)


def _check_orbitals_sampled(w, phi, dphi, n=4096, seed=1):
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(w.n_g, n, replace=False))
    p_ref, d_ref = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz[idx])
    it = torch.as_tensor(idx).cuda()
    p = phi[:, it].cpu().numpy()
    d = dphi[:, :, it].cpu().numpy()
    ep = np.linalg.norm(p - p_ref) / np.linalg.norm(p_ref)
    ed = np.linalg.norm(d - d_ref) / np.linalg.norm(d_ref)
    return ep, ed


def test_h50_chain_orbitals_pivots_fit(api):
    w = wl.h50_chain()
    # orbitals with the contractions emulated on the tensor cores (mode 1)
    phi, dphi = _orbitals(api, w, mode=1)
    ep, ed = _check_orbitals_sampled(w, phi, dphi)
    print("H50 orbitals mode 1: relative errors %.2e %.2e" % (ep, ed))
    assert ep < 1e-12 and ed < 1e-12, (ep, ed)
    del phi, dphi
    phi, dphi = _orbitals(api, w)
    ep, ed = _check_orbitals_sampled(w, phi, dphi)
    assert ep < 1e-12 and ed < 1e-12, (ep, ed)
    wt = _cu(w.grid_w)
    # pivots: identical inputs, truncated selection
    n_cut = 500
    piv = api.isdf_points(phi, dphi, wt, n_cut).cpu().numpy()
    phi_h, dphi_h = phi.cpu().numpy(), dphi.cpu().numpy()
    ref = pivots.select(phi_h, dphi_h, w.grid_w, n_cut, keep_L=False)
    assert np.array_equal(piv, ref.pivots)
    # fit at the full N_mu on the GPU's own selection, FP64 on CUDA cores (mode 0)
    # and with the FP64 products emulated on the tensor cores (mode 1: 16 blocks
    # of 128 in each triangular solve)
    piv_full = api.isdf_points(phi, dphi, wt, w.n_mu)
    P = piv_full.cpu().numpy()
    rng = np.random.default_rng(2)
    cols = np.sort(rng.choice(w.n_g, 256, replace=False))
    Gm = fit.grams(phi_h, dphi_h, P)
    phiP = phi_h[:, P].T
    G = phiP @ phi_h[:, cols]
    B = [G * G] + [(dphi_h[c][:, P].T @ dphi_h[c][:, cols]) * G for c in range(3)]
    it = torch.as_tensor(cols).cuda()
    for mode, fwd_factor in ((0, 8.0), (1, 64.0)):
        xi, xig, jit = api.isdf_fit(phi, dphi, piv_full, fit_mode=mode)
        X = [xi[:, it].cpu().numpy()] + [xig[c][:, it].cpu().numpy() for c in range(3)]
        del xi, xig
        for c in range(4):
            A = Gm[c] + jit[c] * np.eye(len(P))
            back = np.linalg.norm(A @ X[c] - B[c]) / (np.linalg.norm(A) * np.linalg.norm(X[c]))
            Xo = sla.cho_solve(sla.cho_factor(A, lower=True), B[c])
            kappa = np.linalg.cond(A)
            fwd = np.linalg.norm(X[c] - Xo) / np.linalg.norm(Xo)
            print("H50 fit mode %d channel %d: backward %.2e, forward %.2e, cond %.2e, jitter %.1e"
                  % (mode, c, back, fwd, kappa, jit[c]))
            assert back < 1e-10, (mode, c, back)
            assert fwd < max(1e-10, fwd_factor * kappa * np.finfo(float).eps), (mode, c, fwd, kappa)


def test_benzene_orbitals_and_pivots(api):
    w = wl.benzene_c6h6()
    phi, dphi = _orbitals(api, w)
    ep, ed = _check_orbitals_sampled(w, phi, dphi, n=2048)
    assert ep < 1e-12 and ed < 1e-12, (ep, ed)
    n_cut = 200
    piv = api.isdf_points(phi, dphi, _cu(w.grid_w), n_cut).cpu().numpy()
    ref = pivots.select(phi.cpu().numpy(), dphi.cpu().numpy(), w.grid_w, n_cut, keep_L=False)
    assert np.array_equal(piv, ref.pivots)
    del phi, dphi
    torch.cuda.empty_cache()
