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
