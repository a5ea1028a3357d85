"""Pins of the VMC oracle (Sec. II.C: Eqs. Eloc, var-loss, gn) against finite
differences, closed forms and a hand-worked objective."""
import numpy as np
import pytest

from synth import workloads as wl
from oracle import vmc, orbitals, jastrow


def _tiny(n_atom=2, seed=3):
    w = wl.tiny_chain(n_atom=n_atom, n_rad=4, n_ang=6, shells=(0, 1), seed=seed, n_mu=8,
                      jkind="bh", jterms=wl.bh_terms_c4()[:6])
    return w


def test_ao_laplacian_fd():
    w = _tiny()
    pts = np.random.default_rng(0).normal(size=(7, 3)) * 1.2
    lap = vmc.ao_laplacian(w.basis, pts)
    h = 1e-4
    v0, _ = orbitals.eval_ao(w.basis, pts)
    fd = np.zeros_like(lap)
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        vp, _ = orbitals.eval_ao(w.basis, pts + e)
        vm, _ = orbitals.eval_ao(w.basis, pts - e)
        fd += (vp + vm - 2.0 * v0) / (h * h)
    assert np.max(np.abs(fd - lap)) < 1e-5 * max(1.0, np.max(np.abs(lap)))


@pytest.mark.parametrize("with_chi", [False, True])
def test_jastrow_laplacian_fd(with_chi):
    atoms, xyz = wl.h_chain(3, 1.8)
    jas = wl.bh_jastrow(atoms, xyz, wl.bh_terms_c4(), np.random.default_rng(5), scale=0.3)
    jas.b = np.array([1.2])
    jas.d = 0.9
    if with_chi:
        jas = wl.with_chi(jas, [1.0], 6, beta=1.1)
    rng = np.random.default_rng(2)
    ri = rng.normal(size=(5, 3)) * 1.5
    rj = rng.normal(size=(4, 3)) * 1.5
    lap = vmc.lap1_u(ri, rj, jas)
    h = 1e-4
    u0 = jastrow.u_value(ri, rj, jas)
    fd = np.zeros_like(u0)
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        fd += (jastrow.u_value(ri + e, rj, jas) + jastrow.u_value(ri - e, rj, jas) - 2 * u0) / h ** 2
    assert np.max(np.abs(fd - lap)) < 2e-5 * max(1.0, np.max(np.abs(lap)))


def test_local_energy_matches_fd_of_log_psi():
    """E_loc = -1/2 sum_i (lap_i log Psi + |grad_i log Psi|^2) + V with Psi =
    det_up det_down exp(tau), all derivatives by central differences of log|Psi|
    from the orbital values and u alone (no analytic gradient or Laplacian)."""
    w = _tiny(n_atom=2)
    c_occ = w.mo_coef[:, :w.n_occ]
    jas = w.jastrow
    jas.coef = jas.coef * 4.0
    nuc = w.xyz
    Z = np.ones(len(w.atoms))
    n_occ = c_occ.shape[1]
    N = 2 * n_occ
    R = np.random.default_rng(9).normal(size=(N, 3)) * 1.2

    def logpsi(Rx):
        v, _ = orbitals.eval_ao(w.basis, Rx)
        phi = c_occ.T @ v
        ld = 0.0
        for s in range(2):
            idx = np.arange(s * n_occ, (s + 1) * n_occ)
            ld += np.log(abs(np.linalg.det(phi[:, idx].T)))
        U = jastrow.u_value(Rx, Rx, jas)
        iu = np.triu_indices(N, 1)
        return ld + np.sum(U[iu])

    h = 1e-4
    l0 = logpsi(R)
    kin = 0.0
    for i in range(N):
        g2, lap = 0.0, 0.0
        for ax in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, ax] += h
            Rm[i, ax] -= h
            lp, lm = logpsi(Rp), logpsi(Rm)
            g2 += ((lp - lm) / (2 * h)) ** 2
            lap += (lp + lm - 2 * l0) / h ** 2
        kin += -0.5 * (lap + g2)
    V = 0.0
    for i in range(N):
        for j in range(i + 1, N):
            V += 1.0 / np.linalg.norm(R[i] - R[j])
        for I in range(len(Z)):
            V -= Z[I] / np.linalg.norm(R[i] - nuc[I])
    for I in range(len(Z)):
        for K in range(I + 1, len(Z)):
            V += Z[I] * Z[K] / np.linalg.norm(nuc[I] - nuc[K])
    ref = kin + V
    got = vmc.local_energy(R, w.basis, c_occ, jas, nuc, Z)
    assert abs(got - ref) < 1e-5 * max(1.0, abs(ref)), (got, ref)


def test_metropolis_samples_the_reference_density():
    """Two electrons in one s Gaussian exp(-a r^2): |Phi_0|^2 factorises into
    exp(-2 a r_i^2), so <x^2> = 1/(4a) for every coordinate."""
    import dataclasses
    a = 0.7
    basis = wl.Basis(center=np.zeros((1, 3)), powers=np.zeros((1, 3), np.int32),
                     exps=np.array([[a]]), coefs=np.array([[1.0]]), atom=np.zeros(1, np.int32))
    c_occ = np.ones((1, 1))
    rng = np.random.default_rng(4)
    Nw, S = 400, 60
    W = rng.normal(size=(Nw, 2, 3)) * 0.5
    normals = rng.standard_normal((S, 2, Nw, 3))
    uniforms = rng.random((S, 2, Nw))
    W, acc = vmc.metropolis(W, basis, c_occ, normals, uniforms, sigma=0.9)
    x2 = np.mean(W ** 2)
    assert 0.2 < acc / (S * 2 * Nw) < 0.95
    assert abs(x2 - 1.0 / (4 * a)) < 0.06 * (1.0 / (4 * a)), x2


def test_clipped_objective_hand_worked():
    """E = 19 zeros and one 100: mean 5, mean absolute deviation (19*5 + 95)/20 =
    9.5, upper bound 5 + 47.5 = 52.5, so the clipped mean is 52.5/20 = 2.625 and
    the unbiased variance (19 * 2.625^2 + 49.875^2)/19."""
    E = np.array([0.0] * 19 + [100.0])
    Ec, mean, var = vmc.clipped_objective(E)
    assert Ec[-1] == 52.5 and np.all(Ec[:-1] == 0.0)
    assert abs(mean - 2.625) < 1e-15
    assert abs(var - (19 * 2.625 ** 2 + 49.875 ** 2) / 19) < 1e-12


def test_gauss_newton_step_is_least_squares_on_a_linear_model():
    """For E_k(theta) = a_k + B^T theta (no clipping) the variance is a quadratic
    whose minimiser is the least-squares solution of (B - mean B)^T theta =
    -(a - mean a); the step with lambda = 0 and eta = (N_w - 1)/(2 N_w) lands on it."""
    rng = np.random.default_rng(6)
    Nw, P = 200, 4
    a = rng.normal(size=Nw) * 0.1
    B = rng.normal(size=(P, Nw))
    step = vmc.gauss_newton_step(a, B, 0.0, (Nw - 1) / (2 * Nw))
    Bc = B - B.mean(axis=1)[:, None]
    ref, *_ = np.linalg.lstsq(Bc.T, -(a - a.mean()), rcond=None)
    assert np.allclose(step, ref, rtol=1e-10, atol=1e-12)


def gaussian_helium_like(a=0.7, Z=2.0):
    """One s-Gaussian exp(-a r^2) at the origin, doubly occupied, no
    correlator (cusp off, no terms): Phi_0 = phi(r_1) phi(r_2)."""
    basis = wl.Basis(center=np.zeros((1, 3)), powers=np.zeros((1, 3), np.int32),
                     exps=np.array([[a]]), coefs=np.array([[1.0]]), atom=np.zeros(1, np.int32))
    jas = wl.Jastrow(nuc_xyz=np.zeros((1, 3)), nuc_type=np.zeros(1, np.int32),
                     mno=np.zeros((0, 3), np.int32), coef=np.zeros((1, 0)), b=np.ones(1), d=1.0,
                     cusp=False)
    return basis, np.ones((1, 1)), jas, np.zeros((1, 3)), np.array([Z])


def gaussian_helium_like_eloc(R, a, Z):
    """Closed form: lap exp(-a r^2) / exp(-a r^2) = 4 a^2 r^2 - 6 a, so
    E_loc = -1/2 sum_i (4 a^2 r_i^2 - 6 a) - Z sum_i 1/r_i + 1/r_12."""
    r = np.linalg.norm(R, axis=1)
    return (-0.5 * np.sum(4 * a * a * r * r - 6 * a) - Z * np.sum(1.0 / r)
            + 1.0 / np.linalg.norm(R[0] - R[1]))


def test_local_energy_of_a_gaussian_pair_is_closed_form():
    """Eq. Eloc for Psi_T = Phi_0 (tau = 0) with Phi_0 = phi(r_1) phi(r_2),
    phi a single Gaussian: the orbital Laplacian, the drift and the Coulomb
    terms against the closed form, for several configurations."""
    a, Z = 0.7, 2.0
    basis, C, jas, nuc, charges = gaussian_helium_like(a, Z)
    rng = np.random.default_rng(17)
    for _ in range(6):
        R = rng.normal(size=(2, 3)) * 1.3
        got = vmc.local_energy(R, basis, C, jas, nuc, charges)
        want = gaussian_helium_like_eloc(R, a, Z)
        assert abs(got - want) < 1e-11 * max(1.0, abs(want)), (got, want)


def test_clipped_residual_jacobian_matches_finite_differences():
    """Eq. var-loss with clipping active on both sides: for E(theta) = a + B^T theta
    the central differences of the clipped residuals r = E~ - mean(E~) and of the
    clipped variance equal residual_jacobian and 2/(N_w - 1) dr r.  The bounds
    m +- 5 dev move with theta, so the clipped entries follow their bound."""
    rng = np.random.default_rng(8)
    Nw, P = 300, 3
    a = rng.normal(size=Nw)
    a[:5] = [9.0, -11.0, 8.5, -7.9, 12.0]   # beyond m +- 5 dev
    B = rng.normal(size=(P, Nw)) * 0.3
    th = rng.normal(size=P) * 0.1

    def resid(t):
        Ec, mean, var = vmc.clipped_objective(a + B.T @ t)
        return Ec - mean, var

    E = a + B.T @ th
    Ec, mean, var = vmc.clipped_objective(E)
    assert np.sum(Ec != E) >= 4  # clipping is active
    dr = vmc.residual_jacobian(E, B)
    h = 1e-6
    for p in range(P):
        e = np.zeros(P)
        e[p] = h
        rp, vp = resid(th + e)
        rm, vm = resid(th - e)
        assert np.max(np.abs((rp - rm) / (2 * h) - dr[p])) < 1e-7
        grad = 2.0 / (Nw - 1) * dr[p] @ (Ec - mean)
        assert abs((vp - vm) / (2 * h) - grad) < 1e-7 * max(1.0, abs(grad))


def test_energy_jacobian_fd_against_independent_derivatives():
    """energy_jacobian_fd, the reference for dE_loc/dtheta, against derivatives
    formed here by setting d, b_t and c_tk on the correlator directly (not through
    its parameter vector): every row against a five-point stencil (error O(h^4)),
    and the coefficient block against an exact identity.  u is linear in the
    coefficients c (Eq. bh-u) and E_loc holds tau at most squared (Eq. Eloc), so
    along c -> s c the local energy is a quadratic in s and
    sum_k c_k dE/dc_k = (E(2c) - E(0)) / 2 with no truncation error.  A wrong
    sign, step divisor or row order fails one of the two."""
    import copy
    w = _tiny(n_atom=4, seed=4)
    c_occ = w.mo_coef[:, :w.n_occ]
    jas = copy.deepcopy(w.jastrow)
    jas.coef = jas.coef * 4.0
    jas.b = np.asarray(jas.b, float) * 1.1
    nuc, Z = w.xyz, np.ones(len(w.atoms))
    N = 2 * c_occ.shape[1]
    R = np.random.default_rng(21).normal(size=(3, N, 3)) * 1.3
    J = vmc.energy_jacobian_fd(R, w.basis, c_occ, jas, nuc, Z, h=1e-5)
    T, nt = jas.coef.shape

    def E(j):
        return vmc.local_energies(R, w.basis, c_occ, j, nuc, Z)

    def moved(row, t):
        j = copy.deepcopy(jas)
        j.b = np.array(jas.b, float)
        j.coef = np.array(jas.coef, float)
        if row == 0:
            j.d = jas.d + t
        elif row <= T:
            j.b[row - 1] += t
        else:
            j.coef[(row - 1 - T) // nt, (row - 1 - T) % nt] += t
        return j

    assert J.shape == (1 + T + T * nt, R.shape[0])
    h = 1e-3
    for row in range(J.shape[0]):
        five = (-E(moved(row, 2 * h)) + 8 * E(moved(row, h)) - 8 * E(moved(row, -h))
                + E(moved(row, -2 * h))) / (12 * h)
        assert np.max(np.abs(J[row] - five)) < 1e-6 * max(1.0, np.max(np.abs(five))), row

    j0, j2 = copy.deepcopy(jas), copy.deepcopy(jas)
    j0.coef = np.zeros_like(jas.coef)
    j2.coef = 2.0 * jas.coef
    euler = (E(j2) - E(j0)) / 2.0
    got = jas.coef.ravel() @ J[1 + T:]
    assert np.max(np.abs(got - euler)) < 1e-7 * max(1.0, np.max(np.abs(euler))), (got, euler)
    assert np.max(np.abs(euler)) > 1e-3  # the correlator's coefficients matter here
