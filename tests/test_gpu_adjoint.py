"""GPU adjoint dL/dtheta of the Jastrow kernels against the FP64 oracle, central
finite differences and the autograd wrapper."""
import numpy as np
import pytest
import torch

from synth import workloads as wl
from oracle import orbitals, pivots, fit, adjoint

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_17314_b300 import build
    build.build()
    from paper_2607_17314_b300 import api
    return api


def _case(n_atom=3, n_rad=8, n_ang=12, n_mu=24, seed=17, terms=None, scale=4.0):
    w = wl.tiny_chain(n_atom=n_atom, n_rad=n_rad, n_ang=n_ang, shells=(0, 1), n_mu=n_mu, seed=seed,
                      jkind="bh", jterms=terms or wl.bh_terms_c4())
    w.jastrow.coef = w.jastrow.coef * scale
    w.jastrow.b = np.array([1.1])
    w.jastrow.d = 0.95
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    res = pivots.select(phi, dphi, w.grid_w, w.n_mu)
    xi, xit, _ = fit.fit(phi, dphi, res.pivots)
    Wbar = wl.seeded_matrix((4, w.n_mu, w.n_mu), 77)
    return w, xi, xit, Wbar


def _cu(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def test_adjoint_matches_oracle(api):
    w, xi, xit, Wbar = _case()
    ref = adjoint.grad(w.grid_xyz, w.grid_w, xi, xit, w.jastrow, Wbar)
    J = api.jastrow_from(w.jastrow)
    args = (_cu(w.grid_xyz), _cu(w.grid_w), _cu(xi), _cu(xit), J, _cu(Wbar))
    g64 = api.tc_kernel_adjoint(*args, precision="fp64").cpu().numpy()
    g32 = api.tc_kernel_adjoint(*args, precision="fp32").cpu().numpy()
    assert len(ref) == 30
    assert np.linalg.norm(g64 - ref) < 1e-10 * np.linalg.norm(ref), (g64, ref)
    err32 = np.linalg.norm(g32 - ref) / np.linalg.norm(ref)
    print("fp32 adjoint rel err", err32)
    assert err32 < 1e-4


def test_adjoint_with_one_body_term_matches_oracle(api):
    """With the one-body term of Eq. tau-def (parameter-free, in K_c of the
    M^sq factor), FP64 at 1e-10 and FP32 at 1e-4 against the oracle."""
    w, xi, xit, Wbar = _case(n_mu=16, seed=5)
    jas = wl.with_chi(w.jastrow, [1.0], 2 * w.n_occ, beta=0.9)
    ref = adjoint.grad(w.grid_xyz, w.grid_w, xi, xit, jas, Wbar)
    ref0 = adjoint.grad(w.grid_xyz, w.grid_w, xi, xit, w.jastrow, Wbar)
    assert np.linalg.norm(ref - ref0) > 1e-3 * np.linalg.norm(ref)
    args = (_cu(w.grid_xyz), _cu(w.grid_w), _cu(xi), _cu(xit), api.jastrow_from(jas), _cu(Wbar))
    g64 = api.tc_kernel_adjoint(*args, precision="fp64").cpu().numpy()
    g32 = api.tc_kernel_adjoint(*args, precision="fp32").cpu().numpy()
    assert np.linalg.norm(g64 - ref) < 1e-10 * np.linalg.norm(ref)
    assert np.linalg.norm(g32 - ref) < 1e-4 * np.linalg.norm(ref)


def test_adjoint_matches_fd_of_gpu_forward(api):
    """Central differences (h = 1e-4) of L(theta) evaluated with the FP64 GPU
    forward build, for every parameter."""
    w, xi, xit, Wbar = _case(n_atom=2, n_rad=6, n_ang=10, n_mu=12, seed=3)
    J = api.jastrow_from(w.jastrow)
    g, wt, X, Xt, Wb = _cu(w.grid_xyz), _cu(w.grid_w), _cu(xi), _cu(xit), _cu(Wbar)
    g32 = api.tc_kernel_adjoint(g, wt, X, Xt, J, Wb, "fp32").cpu().numpy()
    th = np.concatenate([[J.d, J.b[0]], [J.coef[0][k] for k in range(J.n_terms)]])
    h = 1e-4
    fd = np.zeros_like(th)
    for p in range(len(th)):
        vals = []
        for s in (+1, -1):
            tp = th.copy()
            tp[p] += s * h
            W, _ = api.tc_kernel_build(g, wt, X, Xt, api.jastrow_with_theta(J, tp), "fp64")
            vals.append(float((W * Wb).sum()))
        fd[p] = (vals[0] - vals[1]) / (2 * h)
    assert np.linalg.norm(g32 - fd) < 1e-4 * np.linalg.norm(fd), (g32, fd)


def test_autograd_function(api):
    w, xi, xit, Wbar = _case(n_atom=2, n_rad=6, n_ang=10, n_mu=12, seed=3)
    J = api.jastrow_from(w.jastrow)
    theta = torch.tensor([J.d, J.b[0]] + [J.coef[0][k] for k in range(J.n_terms)],
                         dtype=torch.float64, requires_grad=True)
    W = api.TCKernel.apply(theta, _cu(w.grid_xyz), _cu(w.grid_w), _cu(xi), _cu(xit), J, "fp64")
    loss = (W * _cu(Wbar)).sum()
    loss.backward()
    ref = adjoint.grad(w.grid_xyz, w.grid_w, xi, xit, w.jastrow, Wbar)
    assert np.linalg.norm(theta.grad.numpy() - ref) < 1e-10 * np.linalg.norm(ref)


def test_adjoint_rejects_two_types(api):
    from paper_2607_17314_b300 import _capi as C
    atoms, xyz = wl.benzene()
    jas = wl.bh_jastrow(atoms, xyz, wl.BH_TERMS_C3, np.random.default_rng(0))
    w, xi, xit, Wbar = _case()
    with pytest.raises(C.IsdfError) as e:
        api.tc_kernel_adjoint(_cu(w.grid_xyz), _cu(w.grid_w), _cu(xi), _cu(xit),
                              api.jastrow_from(jas), _cu(Wbar), "fp32")
    assert e.value.status == C.ISDF_E_UNSUPPORTED


def test_adjoint_h20_full_size_on_outer_slices(api):
    """The adjoint at the H20-chain size (40,000 points, N_mu = 800, the 28-term
    one-type correlator: 30 parameters) on outer-grid slices: FP64 adjoint
    against central differences (h = 1e-4) of the FP64 forward over the same
    slice for five sampled parameters, FP32 against FP64, and additivity over
    slices.  xi, xi~ and the seed Wbar are seeded normal samples."""
    w = wl.h20_chain_bh()
    n_g, n_mu = w.grid_xyz.shape[0], w.n_mu
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4321)
    g, wt = _cu(w.grid_xyz), _cu(w.grid_w)
    X = torch.randn((n_mu, n_g), dtype=torch.float64, device="cuda", generator=gen) * 1e-3
    Xt = torch.randn((3, n_mu, n_g), dtype=torch.float64, device="cuda", generator=gen) * 1e-3
    Wb = _cu(wl.seeded_matrix((4, n_mu, n_mu), 77))
    J = api.jastrow_from(w.jastrow)
    g0, g1 = 20000, 20192
    g64 = api.tc_kernel_adjoint(g, wt, X, Xt, J, Wb, "fp64", g_begin=g0, g_end=g1).cpu().numpy()
    g32 = api.tc_kernel_adjoint(g, wt, X, Xt, J, Wb, "fp32", g_begin=g0, g_end=g1).cpu().numpy()
    assert len(g64) == 30
    err32 = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
    a = api.tc_kernel_adjoint(g, wt, X, Xt, J, Wb, "fp64", g_begin=g0, g_end=g0 + 80)
    b = api.tc_kernel_adjoint(g, wt, X, Xt, J, Wb, "fp64", g_begin=g0 + 80, g_end=g1)
    add = float(torch.linalg.norm(a + b - torch.as_tensor(g64).cuda())) / np.linalg.norm(g64)
    th = np.concatenate([[J.d, J.b[0]], [J.coef[0][k] for k in range(J.n_terms)]])
    h = 1e-4
    sample = [0, 1, 2, 15, 29]
    fd = []
    for p in sample:
        vals = []
        for s in (+1, -1):
            tp = th.copy()
            tp[p] += s * h
            W, _ = api.tc_kernel_build(g, wt, X, Xt, api.jastrow_with_theta(J, tp), "fp64",
                                       g_begin=g0, g_end=g1)
            vals.append(float((W * Wb).sum()))
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    efd = np.linalg.norm(g64[sample] - fd) / np.linalg.norm(fd)
    print("H20 slice: FP64 adjoint vs central differences %.2e, FP32 vs FP64 %.2e, "
          "slice additivity %.2e" % (efd, err32, add))
    assert efd < 1e-6
    assert err32 < 1e-4
    assert add < 1e-12
