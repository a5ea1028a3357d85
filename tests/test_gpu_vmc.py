"""GPU VMC optimisation of the correlator (Sec. II.C: Eqs. Eloc, var-loss, gn)
against the FP64 oracle: local energies, their parameter Jacobian, the
Metropolis sampler and the Gauss-Newton step."""
import numpy as np
import pytest
import torch

from synth import workloads as wl
from oracle import vmc, adjoint

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_17314_b300 import build
    build.build()
    from paper_2607_17314_b300 import api
    return api


def _cu(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _basis(b):
    return (_cu(b.center), _cu(b.powers.astype(np.int32)), _cu(b.exps), _cu(b.coefs))


def _system(n_atom=4, n_occ=2, seed=11, n_terms=6, scale=0.3, chi=False):
    atoms, xyz, basis, C, _, jas = wl.vmc_chain(n_atom, seed=seed, terms=wl.bh_terms_c4()[:n_terms],
                                                jscale=scale)
    jas.b = np.array([1.15])
    jas.d = 0.9
    if chi:
        jas = wl.with_chi(jas, [-0.4], 2 * n_occ, beta=1.3)
    return xyz, basis, C, n_occ, jas, np.ones(n_atom)


def _scale(x):
    return max(1.0, float(np.max(np.abs(x))))


@pytest.mark.parametrize("n_atom,n_occ,n_terms,chi", [(4, 2, 6, False), (4, 3, 6, True),
                                                      (3, 1, 0, False), (10, 9, 10, True)])
def test_local_energy_matches_oracle(api, n_atom, n_occ, n_terms, chi):
    xyz, basis, C, n_occ, jas, Z = _system(n_atom, n_occ, n_terms=n_terms, chi=chi)
    if n_terms == 0:
        jas = wl.radial_jastrow(xyz, d=0.8)
    R = wl.vmc_walkers(xyz, 13, 2 * n_occ, seed=5)
    ref = vmc.local_energies(R, basis, C[:, :n_occ], jas, xyz, Z)
    E = api.isdf_vmc_local_energy(_basis(basis), _cu(C), n_occ, _cu(R), api.jastrow_from(jas), Z,
                                  grad=False).cpu().numpy()
    err = np.max(np.abs(E - ref))
    print("E_loc max err", err, "scale", _scale(ref))
    assert err < 1e-10 * _scale(ref), (E, ref)


@pytest.mark.parametrize("case", ["two_types", "high_exponents", "forty_nuclei"])
def test_local_energy_and_jacobian_layouts(api, case):
    """Two nucleus types (benzene geometry), exponents above 3 (the general
    moment table), and more nuclei than lanes (several passes per warp)."""
    if case == "two_types":
        w = wl.benzene_small(n_rad=2, n_ang=6, n_mu=8)
        xyz, basis, C, n_occ, jas = w.xyz, w.basis, w.mo_coef, 5, w.jastrow
        jas.coef = jas.coef * 6.0
        Z = np.array([6.0 if a == "C" else 1.0 for a in w.atoms])
    elif case == "high_exponents":
        xyz, basis, C, n_occ, jas, Z = _system(n_atom=5, n_occ=3, n_terms=0)
        terms = [(4, 1, 2), (0, 5, 0), (2, 6, 3), (1, 1, 1), (8, 0, 0), (3, 3, 4)]
        jas = wl.bh_jastrow(["H"] * 5, xyz, terms, np.random.default_rng(4), scale=0.4)
        jas.b = np.array([1.3])
    else:
        xyz, basis, C, n_occ, jas, Z = _system(n_atom=40, n_occ=3, n_terms=5)
    R = wl.vmc_walkers(xyz, 3, 2 * n_occ, seed=12, spread=1.3)
    h = 1e-5
    refE = vmc.local_energies(R, basis, C[:, :n_occ], jas, xyz, Z)
    refJ = vmc.energy_jacobian_fd(R, basis, C[:, :n_occ], jas, xyz, Z, h=h)
    E, dE = api.isdf_vmc_local_energy(_basis(basis), _cu(C), n_occ, _cu(R), api.jastrow_from(jas),
                                      Z, fd_step=h)
    E, dE = E.cpu().numpy(), dE.cpu().numpy()
    print(case, "E err", np.max(np.abs(E - refE)), "J err", np.max(np.abs(dE - refJ)))
    assert np.max(np.abs(E - refE)) < 1e-10 * _scale(refE), (E, refE)
    tol = 50 * np.finfo(float).eps * _scale(refE) / h
    assert np.max(np.abs(dE - refJ)) < tol, (dE, refJ, tol)


def test_local_energy_many_electrons_per_spin(api):
    """33 electrons per spin: the pivot search spans two rows per lane."""
    xyz, basis, C, _, jas, Z = _system(n_atom=12, n_occ=33, n_terms=3)
    R = wl.vmc_walkers(xyz, 3, 66, seed=8, spread=1.5)
    ref = vmc.local_energies(R, basis, C[:, :33], jas, xyz, Z)
    E = api.isdf_vmc_local_energy(_basis(basis), _cu(C), 33, _cu(R), api.jastrow_from(jas), Z,
                                  grad=False).cpu().numpy()
    assert np.max(np.abs(E - ref)) < 1e-8 * _scale(ref), (E, ref)


def test_local_energy_largest_walker(api):
    """64 electrons per spin (the limit) on 30 nuclei: the pair-factor table no
    longer fits shared memory and the kernel recomputes the pair factors per
    lane.  The seeded configuration keeps both determinants well conditioned
    (condition numbers below 1e4), so FP64 rounding stays near 1e-12."""
    xyz, basis, C, _, jas, Z = _system(n_atom=30, n_occ=64, n_terms=3)
    R = wl.vmc_walkers(xyz, 2, 128, seed=12, spread=0.8)
    h = 1e-5
    refE = vmc.local_energies(R, basis, C[:, :64], jas, xyz, Z)
    refJ = vmc.energy_jacobian_fd(R, basis, C[:, :64], jas, xyz, Z, h=h)
    E, dE = api.isdf_vmc_local_energy(_basis(basis), _cu(C), 64, _cu(R), api.jastrow_from(jas), Z,
                                      fd_step=h)
    E, dE = E.cpu().numpy(), dE.cpu().numpy()
    print("N=128 E err", np.max(np.abs(E - refE)), "J err", np.max(np.abs(dE - refJ)),
          "scales", _scale(refE), _scale(refJ))
    assert np.max(np.abs(E - refE)) < 1e-9 * _scale(refE), (E, refE)
    assert np.max(np.abs(dE - refJ)) < 50 * np.finfo(float).eps * _scale(refE) / h


@pytest.mark.parametrize("chi", [False, True])
def test_jacobian_matches_oracle(api, chi):
    """d and b rows: central differences of the same step on both sides; the
    coefficient rows exact on the GPU against the oracle's central differences
    (exact for a quadratic up to rounding)."""
    xyz, basis, C, n_occ, jas, Z = _system(chi=chi)
    R = wl.vmc_walkers(xyz, 5, 2 * n_occ, seed=21)
    h = 1e-5
    refE = vmc.local_energies(R, basis, C[:, :n_occ], jas, xyz, Z)
    refJ = vmc.energy_jacobian_fd(R, basis, C[:, :n_occ], jas, xyz, Z, h=h)
    E, dE = api.isdf_vmc_local_energy(_basis(basis), _cu(C), n_occ, _cu(R), api.jastrow_from(jas),
                                      Z, fd_step=h)
    E, dE = E.cpu().numpy(), dE.cpu().numpy()
    assert dE.shape == refJ.shape
    assert np.max(np.abs(E - refE)) < 1e-9 * _scale(refE)
    err = np.max(np.abs(dE - refJ), axis=1)
    print("Jacobian row errors", err)
    # central differences of step h carry rounding ~ eps |E| / h on either side
    tol = 50 * np.finfo(float).eps * _scale(refE) / h
    assert np.all(err < tol), (dE, refJ, tol)


def test_theta_from_device_overrides_struct(api):
    xyz, basis, C, n_occ, jas, Z = _system()
    th = adjoint.get_theta(jas)
    th2 = th * (1.0 + 0.1 * np.sin(np.arange(len(th))))
    jas2 = adjoint.set_theta(jas, th2)
    R = wl.vmc_walkers(xyz, 7, 2 * n_occ, seed=3)
    ref = vmc.local_energies(R, basis, C[:, :n_occ], jas2, xyz, Z)
    E = api.isdf_vmc_local_energy(_basis(basis), _cu(C), n_occ, _cu(R), api.jastrow_from(jas), Z,
                                  theta=_cu(th2), grad=False).cpu().numpy()
    assert np.max(np.abs(E - ref)) < 1e-9 * _scale(ref)


@pytest.mark.parametrize("n_occ,n_steps", [(2, 4), (3, 3)])
def test_sampler_matches_oracle(api, n_occ, n_steps):
    """Same random numbers -> the same accepted moves (exact count) and final
    positions; the GPU takes the ratio against an updated inverse, the oracle
    from two determinants."""
    xyz, basis, C, _, jas, Z = _system(n_atom=4, n_occ=n_occ)
    N, Nw = 2 * n_occ, 6
    R = wl.vmc_walkers(xyz, Nw, N, seed=31)
    normals, uniforms = wl.vmc_random(n_steps, N, Nw, seed=32)
    refR, ref_acc = vmc.metropolis(R, basis, C[:, :n_occ], normals, uniforms, 0.6)
    Rg = _cu(R)
    acc = api.isdf_vmc_sample(_basis(basis), _cu(C), n_occ, Rg, _cu(normals), _cu(uniforms), 0.6)
    assert acc == ref_acc
    assert 0 < acc < n_steps * N * Nw
    assert np.max(np.abs(Rg.cpu().numpy() - refR)) < 1e-12


def test_gn_step_matches_oracle(api):
    rng = np.random.default_rng(41)
    Nw, P = 400, 9
    E = -2.0 + 0.3 * rng.standard_normal(Nw)
    E[:4] = [8.0, -12.0, 6.5, -9.0]           # beyond m +- 5 dev: both clip branches
    dE = rng.standard_normal((P, Nw))
    dE[2] *= 0.01
    lam, eta = 1e-3, 0.7
    ref = vmc.gauss_newton_step(E, dE, lam, eta)
    _, mean, var = vmc.clipped_objective(E)
    theta = _cu(np.arange(P, dtype=float))
    step, stats = api.isdf_vmc_gn_step(_cu(E), _cu(dE), lam, eta, theta=theta)
    step, stats = step.cpu().numpy(), stats.cpu().numpy()
    assert np.max(np.abs(step - ref)) < 1e-10 * np.max(np.abs(ref)), (step, ref)
    assert abs(stats[0] - mean) < 1e-12 and abs(stats[1] - var) < 1e-12 * var
    assert np.max(np.abs(theta.cpu().numpy() - (np.arange(P) + step))) == 0.0


def test_objective_matches_oracle(api):
    rng = np.random.default_rng(44)
    E = -1.0 + 0.5 * rng.standard_normal(300)
    E[7], E[9] = 15.0, -20.0
    _, mean, var = vmc.clipped_objective(E)
    m = np.mean(E)
    dev = np.mean(np.abs(E - m))
    st = api.isdf_vmc_objective(_cu(E)).cpu().numpy()
    assert np.allclose(st, [mean, var, m, dev], rtol=1e-13, atol=1e-14), (st, mean, var, m, dev)


def test_optimisation_lowers_the_sampled_variance(api):
    """Sample |Phi_0|^2, then Gauss-Newton iterations on that fixed sample
    (the reference-variance protocol) with the adaptive shift: the clipped
    variance never rises and ends well below its start."""
    xyz, basis, C, n_occ, jas, Z = _system(n_atom=6, n_occ=3, n_terms=10, scale=0.2)
    N, Nw = 2 * n_occ, 512
    Rg = _cu(wl.vmc_walkers(xyz, Nw, N, seed=51))
    normals, uniforms = wl.vmc_random(20, N, Nw, seed=52)
    B = _basis(basis)
    api.isdf_vmc_sample(B, _cu(C), n_occ, Rg, _cu(normals), _cu(uniforms), 0.5)
    J = api.jastrow_from(jas)
    theta = _cu(adjoint.get_theta(jas))
    opt = api.VmcOptimizer(B, _cu(C), n_occ, Rg, J, Z, theta)
    v0 = opt.var
    hist = [opt.step() for _ in range(8)]
    var = [v0] + [h[0] for h in hist]
    print("variance per iteration", var, "lambda", [h[1] for h in hist])
    assert np.all(np.isfinite(var)) and np.all(np.diff(var) <= 0.0)
    assert var[-1] < 0.8 * var[0]
    # the final theta reproduces the final variance
    E = api.isdf_vmc_local_energy(B, _cu(C), n_occ, Rg, J, Z, theta=theta, grad=False)
    assert float(api.isdf_vmc_objective(E)[1]) == var[-1]


def test_polyak_running_mean(api):
    """The running mean of six iterates; the first call copies theta without
    reading avg, so avg may start as anything (NaN, 1e300 here)."""
    rng = np.random.default_rng(61)
    xs = rng.standard_normal((6, 11))
    avg = _cu(np.where(np.arange(11) % 2 == 0, np.nan, 1e300))
    api.isdf_vmc_polyak(_cu(xs[0]), avg, 1)
    assert np.array_equal(avg.cpu().numpy(), xs[0])
    for k, x in enumerate(xs, 1):
        api.isdf_vmc_polyak(_cu(x), avg, k)
    assert np.allclose(avg.cpu().numpy(), xs.mean(axis=0), rtol=1e-14, atol=1e-15)


def test_schedule_with_fresh_samples_and_averaging(api):
    """Warm-up and refinement steps, each on a continued Metropolis sample of
    |Phi_0|^2, then the Polyak-Ruppert average of the refinement tail: the
    averaged correlator has a lower clipped variance than the starting one on
    a fresh, independent sample."""
    xyz, basis, C, n_occ, jas, Z = _system(n_atom=6, n_occ=3, n_terms=10, scale=0.2)
    N, Nw = 2 * n_occ, 512
    B = _basis(basis)
    Cg = _cu(C)
    J = api.jastrow_from(jas)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(71)
    Rg = _cu(wl.vmc_walkers(xyz, Nw, N, seed=72))
    nrm = torch.randn((20, N, Nw, 3), dtype=torch.float64, device="cuda", generator=gen)
    uni = torch.rand((20, N, Nw), dtype=torch.float64, device="cuda", generator=gen)
    api.isdf_vmc_sample(B, Cg, n_occ, Rg, nrm, uni, 0.5)          # burn-in
    theta0 = _cu(adjoint.get_theta(jas))
    theta = theta0.clone()
    avg, hist = api.vmc_schedule(B, Cg, n_occ, Rg, J, Z, theta, n_warm=4, n_refine=6, window=4,
                                 sweeps=4, sigma=0.5, generator=gen)
    print("schedule", [(round(h[0], 4), h[1], h[2], round(h[3], 3)) for h in hist])
    assert len(hist) == 10 and all(np.isfinite(h[0]) and 0.2 < h[3] < 0.95 for h in hist)
    assert torch.all(torch.isfinite(avg))
    # an independent sample
    R2 = _cu(wl.vmc_walkers(xyz, Nw, N, seed=73))
    nrm = torch.randn((30, N, Nw, 3), dtype=torch.float64, device="cuda", generator=gen)
    uni = torch.rand((30, N, Nw), dtype=torch.float64, device="cuda", generator=gen)
    api.isdf_vmc_sample(B, Cg, n_occ, R2, nrm, uni, 0.5)
    v0 = float(api.isdf_vmc_objective(api.isdf_vmc_local_energy(B, Cg, n_occ, R2, J, Z, theta=theta0,
                                                                grad=False))[1])
    v1 = float(api.isdf_vmc_objective(api.isdf_vmc_local_energy(B, Cg, n_occ, R2, J, Z, theta=avg,
                                                                grad=False))[1])
    print("clipped variance on a fresh sample: start", v0, "averaged", v1)
    assert v1 < v0


def test_local_energy_of_a_gaussian_pair_is_closed_form(api):
    """The GPU kernels against the closed form of E_loc for one doubly
    occupied s-Gaussian exp(-a r^2) at a Z = 2 nucleus and no correlator:
    E_loc = -1/2 sum_i (4 a^2 r_i^2 - 6 a) - Z sum_i 1/r_i + 1/r_12."""
    a, Z = 0.7, 2.0
    basis = wl.Basis(center=np.zeros((1, 3)), powers=np.zeros((1, 3), np.int32),
                     exps=np.array([[a]]), coefs=np.array([[1.0]]), atom=np.zeros(1, np.int32))
    jas = wl.Jastrow(nuc_xyz=np.zeros((1, 3)), nuc_type=np.zeros(1, np.int32),
                     mno=np.zeros((0, 3), np.int32), coef=np.zeros((1, 0)), b=np.ones(1), d=1.0,
                     cusp=False)
    R = np.random.default_rng(23).normal(size=(37, 2, 3)) * 1.3
    E = api.isdf_vmc_local_energy(_basis(basis), _cu(np.ones((1, 1))), 1, _cu(R),
                                  api.jastrow_from(jas), [Z], grad=False).cpu().numpy()
    r = np.linalg.norm(R, axis=2)
    want = (-0.5 * np.sum(4 * a * a * r * r - 6 * a, axis=1) - Z * np.sum(1.0 / r, axis=1)
            + 1.0 / np.linalg.norm(R[:, 0] - R[:, 1], axis=1))
    assert np.max(np.abs(E - want)) < 1e-12 * _scale(want), (E, want)
