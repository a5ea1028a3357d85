"""Stage-1 parity at full workload sizes, on sampled outputs.

The W build runs at the grid and N_mu of the H50-chain workload (radial
correlator, 100,000 points, N_mu = 2000) and of the benzene workload
(multi-centre correlator, 271,800 points, N_mu = 8000) over an outer-grid
slice, in the same kernels and launch shape as the full build (persistent
grid of one CTA per SM; the inner sum spans the whole grid).  Sampled calG
entries are checked against the oracle computed one by one, within 1e-5 of
the normwise bound sum_g' |w_g' xi_nu(g') K_c(g, g')| (the dot-product error
scale); W of the slice is checked against FP64 products of the returned calG.
xi and xi~ are seeded normal samples of the workloads' shapes.
"""
import numpy as np
import pytest
import torch

from synth import workloads as wl
from oracle import jastrow as ojas

pytestmark = pytest.mark.gpu

f64 = torch.float64


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2607_17314_b300 import api
    return api


def _case(name):
    if name == "h50_chain":
        atoms, xyz = wl.h_chain(50, 1.8)
        grid, w = wl.becke_grid(xyz, 40, 50)
        return grid, w, 2000, wl.radial_jastrow(xyz)
    atoms, xyz = wl.benzene()
    grid, w = wl.becke_grid(xyz, 75, 302)
    return grid, w, 8000, wl.bh_jastrow(atoms, xyz, wl.BH_TERMS_C3, np.random.default_rng(3001))


@pytest.mark.parametrize("name", ["h50_chain", "benzene"])
def test_full_size_stage1_sampled(P, name):
    grid, w, n_mu, jas = _case(name)
    n_g = grid.shape[0]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(77)
    xi = torch.randn((n_mu, n_g), dtype=f64, device="cuda", generator=gen) * 1e-3
    xig = torch.randn((3, n_mu, n_g), dtype=f64, device="cuda", generator=gen) * 1e-3
    g0 = n_g // 3 + 5          # a slice that starts and ends off the 64-point tiles
    g1 = g0 + 2048 + 21
    gd = torch.tensor(grid, device="cuda")
    wd = torch.tensor(w, device="cuda")
    W, calG = P.tc_kernel_build(gd, wd, xi, xig, P.jastrow_from(jas), "bf16x3",
                                g_begin=g0, g_end=g1)
    rng = np.random.default_rng(5)
    mus = np.sort(rng.choice(n_mu, 4, replace=False))
    gs = np.sort(rng.choice(np.arange(g0, g1), 3, replace=False))
    wx = xi[torch.as_tensor(mus, device="cuda")].cpu().numpy() * w[None, :]
    K = ojas.kernels(grid[gs], grid, jas, gs, np.arange(n_g))        # [4, 3, n_g]
    ref = np.einsum("mg,chg->cmh", wx, K)
    bound = np.einsum("mg,chg->cmh", np.abs(wx), np.abs(K))
    got = calG[:, torch.as_tensor(mus, device="cuda")][:, :, torch.as_tensor(gs - g0, device="cuda")]
    got = got.cpu().numpy()
    worst = float(np.max(np.abs(got - ref) / bound))
    print(name, "sampled calG error / normwise bound:", worst)
    assert worst < 1e-5
    for c in range(4):
        src = xig[c] if c < 3 else xi
        Wr = (src[:, g0:g1] * wd[g0:g1]) @ calG[c].T
        err = float(torch.linalg.norm(W[c] - Wr) / torch.linalg.norm(Wr))
        assert err < 1e-5, (c, err)
    del xi, xig, W, calG
    torch.cuda.empty_cache()
