"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here compares the oracle with something other than itself: a
closed form, a finite difference, a brute-force sum, an analytic integral,
a linear-algebra identity, or the paper's pre-ISDF definitions.
"""
import dataclasses
import math

import numpy as np
import pytest

from synth import workloads as wl
from oracle import orbitals, jastrow, pivots, fit, wbuild, xtc, energies


@pytest.fixture(scope="module")
def tiny():
    """3-atom H chain, one s shell per atom: 3 orbitals, 3 x 16 x 26 grid."""
    w = wl.tiny_chain(n_atom=3, n_rad=16, n_ang=26, shells=(0,), n_mu=6, seed=11)
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    return w, phi, dphi


@pytest.fixture(scope="module")
def h6():
    w = wl.h6_chain()
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    return w, phi, dphi


# ---------------------------------------------------------------- orbitals

def test_single_primitive_closed_form():
    """One normalised p_x primitive at a known point against its formula."""
    b = wl.Basis(center=np.array([[0.1, -0.2, 0.3]]), powers=np.array([[1, 0, 0]], np.int32),
                 exps=np.array([[0.7]]), coefs=np.array([[1.3]]), atom=np.zeros(1, np.int32))
    r = np.array([[0.5, 0.4, -0.1]])
    v, g = orbitals.eval_ao(b, r)
    x, y, z = r[0] - b.center[0]
    r2 = x * x + y * y + z * z
    ref = 1.3 * x * math.exp(-0.7 * r2)
    assert abs(v[0, 0] - ref) < 1e-15
    # analytic derivative along x: (1 - 2 a x^2) exp(-a r^2)
    assert abs(g[0, 0, 0] - 1.3 * (1 - 2 * 0.7 * x * x) * math.exp(-0.7 * r2)) < 1e-15
    assert abs(g[1, 0, 0] - 1.3 * x * (-2 * 0.7 * y) * math.exp(-0.7 * r2)) < 1e-15


def test_orbital_gradient_fd(h6):
    w, phi, dphi = h6
    rng = np.random.default_rng(0)
    pts = w.grid_xyz[rng.choice(w.n_g, 40, replace=False)]
    h = 1e-5
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        fp, _ = orbitals.eval_orbitals(w.basis, w.mo_coef, pts + e)
        fm, _ = orbitals.eval_orbitals(w.basis, w.mo_coef, pts - e)
        _, d = orbitals.eval_orbitals(w.basis, w.mo_coef, pts)
        fd = (fp - fm) / (2 * h)
        assert np.max(np.abs(fd - d[ax])) < 1e-7 * max(1.0, np.max(np.abs(d[ax])))


def test_orbitals_match_analytic_overlap():
    """Grid quadrature of phi_p phi_q reproduces the analytic L2 overlap used
    to orthonormalise the orbitals (C^T S_AO C = I), on a fine one-atom grid."""
    w = wl.tiny_chain(n_atom=1, n_rad=80, n_ang=302, shells=(0, 1), seed=3)
    phi, _ = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    ov = (phi * w.grid_w[None, :]) @ phi.T
    assert np.max(np.abs(ov - np.eye(w.n_orb))) < 2e-3


# ---------------------------------------------------------------- Jastrow

def test_radial_closed_form():
    jas = wl.radial_jastrow(np.zeros((2, 3)))
    ri = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, -0.5]])
    rj = np.array([[0.3, -0.4, 1.2], [2.0, 0.0, 0.0]])
    K = jastrow.kernels(ri, rj, jas)
    for a in range(2):
        for b in range(2):
            dv = ri[a] - rj[b]
            r = np.linalg.norm(dv)
            up = 1.0 / (2.0 * (1.0 + r) ** 2)
            assert np.allclose(K[:3, a, b], up * dv / r, rtol=1e-14, atol=0)
            assert abs(K[3, a, b] - 1.0 / (4.0 * (1.0 + r) ** 4)) < 1e-15
    u = jastrow.u_value(ri, rj, jas)
    r = np.linalg.norm(ri[1] - rj[0])
    assert abs(u[1, 0] - r / (2 * (1 + r))) < 1e-15


@pytest.mark.parametrize("terms", [wl.BH_TERMS_C3, wl.bh_terms_c4()])
def test_bh_gradient_fd(terms):
    atoms, xyz = wl.benzene() if len(terms) == 10 else wl.h_chain(4, 1.8)
    jas = wl.bh_jastrow(atoms, xyz, terms, np.random.default_rng(5), scale=0.3)
    jas.b = np.linspace(0.8, 1.3, jas.n_types)
    jas.d = 1.1
    rng = np.random.default_rng(1)
    ri = rng.normal(size=(7, 3)) * 2
    rj = rng.normal(size=(5, 3)) * 2
    g = jastrow.grad1_u(ri, rj, jas)
    h = 1e-6
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        fd = (jastrow.u_value(ri + e, rj, jas) - jastrow.u_value(ri - e, rj, jas)) / (2 * h)
        assert np.max(np.abs(fd - g[ax])) < 1e-8


def test_bh_symmetry_and_cusp():
    atoms, xyz = wl.h_chain(3, 1.8)
    jas = wl.bh_jastrow(atoms, xyz, wl.bh_terms_c4(), np.random.default_rng(2), scale=0.3)
    rng = np.random.default_rng(3)
    a = rng.normal(size=(6, 3))
    b = rng.normal(size=(6, 3))
    assert np.allclose(jastrow.u_value(a, b, jas), jastrow.u_value(b, a, jas).T, rtol=1e-13)
    # opposite-spin Kato: du/dr12 -> 1/2 as r12 -> 0 (no free term has o = 1)
    p = np.array([[0.2, 0.1, 0.3]])
    e = np.array([[0.0, 0.0, 1.0]])
    # symmetric displacement keeps the e-n terms fixed to first order
    r = 1e-6
    slope = (jastrow.u_value(p + 0.5 * r * e, p - 0.5 * r * e, jas)
             - jastrow.u_value(p, p, jas))[0, 0] / r
    assert abs(slope - 0.5) < 1e-5


def _chi_jastrow(n_elec=6):
    atoms, xyz = wl.h_chain(3, 1.8)
    jas = wl.bh_jastrow(atoms, xyz, wl.bh_terms_c4()[:6], np.random.default_rng(8), scale=0.3)
    return wl.with_chi(jas, [1.0], n_elec, beta=1.3)


def test_chi_one_body_closed_forms():
    """chi(r) = sum_I a r_I/(1 + beta r_I) (the reading of the one-body cusp
    factor): zero on a nucleus of a lone centre, slope a = -Z there (the
    electron-nucleus cusp), limit a/beta far away, and grad chi by central
    differences."""
    jas = wl.with_chi(wl.radial_jastrow(np.zeros((1, 3))), [2.0], 4, beta=0.7)
    e = np.array([[0.3, -0.4, 0.8660254037844386]])
    e /= np.linalg.norm(e)
    assert jastrow.chi_value(np.zeros((1, 3)), jas)[0] == 0.0
    h = 1e-7
    assert abs(jastrow.chi_value(h * e, jas)[0] / h - (-2.0)) < 1e-6
    assert abs(jastrow.chi_value(1e9 * e, jas)[0] - (-2.0 / 0.7)) < 1e-7
    r = 1.7
    assert abs(jastrow.chi_value(r * e, jas)[0] - (-2.0 * r / (1.0 + 0.7 * r))) < 1e-15
    jas3 = _chi_jastrow()
    pts = np.random.default_rng(4).normal(size=(6, 3)) * 2
    g = jastrow.chi_grad(pts, jas3)
    for ax in range(3):
        d = np.zeros(3)
        d[ax] = 1e-6
        fd = (jastrow.chi_value(pts + d, jas3) - jastrow.chi_value(pts - d, jas3)) / 2e-6
        assert np.max(np.abs(fd - g[ax])) < 1e-8


def test_chi_pair_kernel_resums_one_body_term():
    """Eq. tau-def: for N electrons, sum_i chi(r_i) + sum_{i<j} u2(r_i, r_j)
    equals sum_{i<j} u(r_i, r_j) with u = u2 + [chi_i + chi_j]/(N-1); and the
    chi part of grad_1 u summed over the N-1 partners j != i gives grad chi(r_i)
    (the ordered-pair evaluation of the numerical implementation notes)."""
    N = 6
    jas = _chi_jastrow(N)
    import dataclasses
    u2 = dataclasses.replace(jas, chi_a=None, chi_b=None, n_elec=0)
    R = np.random.default_rng(11).normal(size=(N, 3)) * 1.5
    iu = np.triu_indices(N, 1)
    lhs = np.sum(jastrow.chi_value(R, jas)) + np.sum(jastrow.u_value(R, R, u2)[iu])
    rhs = np.sum(jastrow.u_value(R, R, jas)[iu])
    assert abs(lhs - rhs) < 1e-13 * max(1.0, abs(lhs))
    gchi = jastrow.grad1_u(R, R, jas) - jastrow.grad1_u(R, R, u2)   # [3, N, N]
    off = ~np.eye(N, dtype=bool)
    summed = np.stack([np.sum(np.where(off, gchi[ax], 0.0), axis=1) for ax in range(3)])
    h = 1e-6
    for ax in range(3):
        d = np.zeros(3)
        d[ax] = h
        fd = (jastrow.chi_value(R + d, jas) - jastrow.chi_value(R - d, jas)) / (2 * h)
        assert np.max(np.abs(summed[ax] - fd)) < 1e-8


def test_chi_gradient_fd_of_u():
    jas = _chi_jastrow()
    rng = np.random.default_rng(12)
    ri = rng.normal(size=(5, 3)) * 2
    rj = rng.normal(size=(4, 3)) * 2
    g = jastrow.grad1_u(ri, rj, jas)
    h = 1e-6
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        fd = (jastrow.u_value(ri + e, rj, jas) - jastrow.u_value(ri - e, rj, jas)) / (2 * h)
        assert np.max(np.abs(fd - g[ax])) < 1e-8


def test_self_pair_masked():
    jas = wl.radial_jastrow(np.zeros((1, 3)))
    pts = np.random.default_rng(0).normal(size=(5, 3))
    K = jastrow.kernels(pts, pts, jas, np.arange(5), np.arange(5))
    assert np.all(K[:, np.arange(5), np.arange(5)] == 0.0)
    assert np.all(np.isfinite(K))


# ---------------------------------------------------------------- pivots

def _dense_S(phi, dphi, w, grad):
    t1 = phi.T @ phi
    if grad:
        t2 = sum(dphi[c].T @ dphi[c] for c in range(3))
        return np.outer(w, w) * t1 * t2
    return np.outer(w, w) * t1 * t1


def test_first_pivot_is_argmax_of_closed_form(h6):
    w, phi, dphi = h6
    res = pivots.select(phi, dphi, w.grid_w, 1, mode="scalar")
    dens = np.sum(phi * phi, axis=0)
    d0 = w.grid_w ** 2 * dens ** 2
    assert res.piv_s[0] == int(np.argmax(d0))
    res = pivots.select(phi, dphi, w.grid_w, 1, mode="gradient")
    gd = np.sum(dphi * dphi, axis=(0, 1))
    assert res.piv_v[0] == int(np.argmax(w.grid_w ** 2 * dens * gd))


@pytest.mark.parametrize("grad", [False, True])
def test_pivot_columns_match_dense_cholesky(tiny, grad):
    """L = S[:, P] chol(S[P,P])^{-T} and d = diag(S) - rowsum(L^2), from a
    dense S built with numpy."""
    w, phi, dphi = tiny
    k = 5
    res = pivots.select(phi, dphi, w.grid_w, k, mode="gradient" if grad else "scalar")
    P = res.piv_v if grad else res.piv_s
    L = res.L_v if grad else res.L_s
    S = _dense_S(phi, dphi, w.grid_w, grad)
    R = np.linalg.cholesky(S[np.ix_(P, P)])
    Lref = np.linalg.solve(R, S[P, :]).T                  # [n_g, k]
    scale = np.max(np.abs(Lref))
    assert np.max(np.abs(L.T - Lref)) < 1e-9 * scale
    dref = np.diag(S) - np.sum(Lref ** 2, axis=1)
    dref[P] = 0
    assert np.max(np.abs((res.d_v if grad else res.d_s) - np.maximum(dref, 0))) < 1e-9 * np.max(np.diag(S))
    # pivoted Cholesky picks non-increasing pivots
    piv_vals = np.array([L[j, P[j]] for j in range(k)])
    assert np.all(np.diff(piv_vals) <= 1e-12 * piv_vals[0])


def test_scalar_rank_exhausts_at_pair_count(tiny):
    """The scalar matrix has rank n_orb (n_orb + 1) / 2 (distinct pair
    products); the pivot loop stops exactly there."""
    w, phi, dphi = tiny
    n = w.n_orb
    res = pivots.select(phi, dphi, w.grid_w, 50, mode="scalar")
    assert res.rank_exhausted
    assert len(res.piv_s) == n * (n + 1) // 2


def test_fusion_rule(h6):
    w, phi, dphi = h6
    res = pivots.select(phi, dphi, w.grid_w, w.n_mu, mode="fused")
    assert len(res.pivots) == w.n_mu and not res.rank_exhausted
    assert len(set(res.pivots.tolist())) == w.n_mu
    # union in append order: alternate scalar / gradient, skip repeats
    seq = []
    for j in range(max(len(res.piv_s), len(res.piv_v))):
        for lst in (res.piv_s, res.piv_v):
            if j < len(lst) and lst[j] not in seq:
                seq.append(int(lst[j]))
    assert seq[:w.n_mu] == res.pivots.tolist()


# ---------------------------------------------------------------- fit

def test_nystrom_identity(h6):
    """Pivot residual trace = weighted fit residual (scalar channel, same
    pivots): sum_g d_g = sum_g w_g^2 r_g."""
    w, phi, dphi = h6
    res = pivots.select(phi, dphi, w.grid_w, 40, mode="scalar")
    xi, _, lams = fit.fit(phi, dphi, res.piv_s, channels=(0,))
    assert lams[0] == 0.0
    r = fit.fit_residual(phi, w.grid_w, res.piv_s, xi)
    a, b = np.sum(res.d_s), np.sum(r)
    assert abs(a - b) < 1e-8 * np.sum(w.grid_w ** 2 * np.sum(phi * phi, 0) ** 2)
    assert abs(a - b) / abs(a) < 1e-5


def test_interpolation_property(h6):
    w, phi, dphi = h6
    res = pivots.select(phi, dphi, w.grid_w, w.n_mu)
    xi, xit, lams = fit.fit(phi, dphi, res.pivots)
    assert np.all(lams == 0)
    P = res.pivots
    assert np.max(np.abs(xi[:, P] - np.eye(len(P)))) < 1e-7
    for c in range(3):
        assert np.max(np.abs(xit[c][:, P] - np.eye(len(P)))) < 1e-7


def test_full_rank_reconstruction(tiny):
    """At full scalar rank the ISDF reproduces every pair density."""
    w, phi, dphi = tiny
    n = w.n_orb
    res = pivots.select(phi, dphi, w.grid_w, n * (n + 1) // 2, mode="scalar")
    xi, _, _ = fit.fit(phi, dphi, res.piv_s, channels=(0,))
    P = res.piv_s
    for p in range(n):
        for q in range(n):
            rec = (phi[p, P] * phi[q, P]) @ xi
            assert np.max(np.abs(rec - phi[p] * phi[q])) < 1e-8 * np.max(np.abs(phi[p] * phi[q]))


def test_full_rank_gradient_reconstruction(tiny):
    """With both channels run to exhaustion (the fused set spans every
    product phi_p d_c phi_q), the gradient-channel fit reproduces those
    products on the whole grid (Sec. II.D, gradient normal equations)."""
    w, phi, dphi = tiny
    n = w.n_orb
    res = pivots.select(phi, dphi, w.grid_w, 33)
    assert res.rank_exhausted
    P = res.pivots
    _, xit, _ = fit.fit(phi, dphi, P)
    for c in range(3):
        for p in range(n):
            for q in range(n):
                target = phi[p] * dphi[c][q]
                rec = (phi[p, P] * dphi[c][q, P]) @ xit[c]
                assert np.max(np.abs(rec - target)) < 1e-7 * np.max(np.abs(target))


def test_jitter_schedule_on_matrices_with_known_spectra():
    """Adaptive Tikhonov shift of the fit's Cholesky (Sec. IV.B; schedule a
    reading: lambda = 0, then 1e-14 max diag, x10 per retry, 8 retries) on
    2 x 2 matrices [[a, 1], [1, a]] whose eigenvalues a - 1 and a + 1 fix how
    many retries succeed."""
    # exactly singular: the first shift suffices
    L, lam = fit.cholesky_with_jitter(np.array([[1.0, 1.0], [1.0, 1.0]]))
    assert lam == 1e-14
    assert np.allclose(L @ L.T, [[1 + 1e-14, 1.0], [1.0, 1 + 1e-14]], rtol=0, atol=1e-15)
    # lowest eigenvalue -5e-12: shifts 1e-14 a, 1e-13 a, 1e-12 a fail, 1e-11 a succeeds
    a = 1.0 - 5e-12
    _, lam = fit.cholesky_with_jitter(np.array([[a, 1.0], [1.0, a]]))
    assert abs(lam - 1e-11 * a) < 1e-12 * 1e-11
    # positive definite: no shift
    _, lam = fit.cholesky_with_jitter(np.array([[2.0, 1.0], [1.0, 2.0]]))
    assert lam == 0.0
    # indefinite (eigenvalue -1): no shift up to 1e-7 helps
    with pytest.raises(np.linalg.LinAlgError):
        fit.cholesky_with_jitter(np.array([[1.0, 2.0], [2.0, 1.0]]))


# ---------------------------------------------------------------- W

def _geometry_case(seed=21, n_g=150, n_mu=5):
    """Random points and fit functions with a two-type multi-centre
    correlator (b != 1, d != 1), so that nuclei and both scaled distances
    enter every kernel value."""
    rng = np.random.default_rng(seed)
    atoms = ["C", "H", "H"]
    xyz = np.array([[0.0, 0.0, 0.0], [1.1, 0.9, 0.0], [-1.2, 0.4, 0.7]])
    jas = wl.bh_jastrow(atoms, xyz, wl.bh_terms_c4(), rng, scale=0.3, d=1.2)
    jas.b = np.array([0.8, 1.3])
    grid = rng.normal(size=(n_g, 3)) * 1.5
    w = rng.uniform(0.2, 1.0, size=n_g)
    xi = rng.normal(size=(n_mu, n_g))
    xit = rng.normal(size=(3, n_mu, n_g))
    return grid, w, xi, xit, jas


def _moved(jas, f):
    return dataclasses.replace(jas, nuc_xyz=f(jas.nuc_xyz))


def test_w_translation_and_permutation_invariant():
    """W depends on differences of positions only, and the double grid sum
    does not depend on the order of the points (Eqs. K1-isdf, K3-isdf)."""
    grid, w, xi, xit, jas = _geometry_case()
    W, _ = wbuild.build(grid, w, xi, xit, jas, batch=64)
    t = np.array([3.7, -2.2, 0.9])
    Wt, _ = wbuild.build(grid + t, w, xi, xit, _moved(jas, lambda x: x + t), batch=64)
    scale = np.max(np.abs(W))
    assert np.max(np.abs(Wt - W)) < 1e-12 * scale
    perm = np.random.default_rng(5).permutation(grid.shape[0])
    Wp, _ = wbuild.build(grid[perm], w[perm], xi[:, perm], xit[:, :, perm], jas, batch=37)
    assert np.max(np.abs(Wp - W)) < 1e-12 * scale


def test_w_rotation_covariance():
    """Rotating points and nuclei by R rotates the kernel gradient, so with one
    fit function for all three channels u1 turns as a vector,
    u1'^c = sum_d R_cd u1^d, and u3 (a squared norm) is unchanged.  A channel
    computed from the wrong coordinate fails this."""
    grid, w, xi, _, jas = _geometry_case(seed=22)
    xit = np.stack([xi, xi, xi])
    q, _ = np.linalg.qr(np.random.default_rng(8).normal(size=(3, 3)))
    R = q * np.sign(np.linalg.det(q))
    W, _ = wbuild.build(grid, w, xi, xit, jas, batch=64)
    Wr, _ = wbuild.build(grid @ R.T, w, xi, xit, _moved(jas, lambda x: x @ R.T), batch=64)
    scale = np.max(np.abs(W))
    assert np.max(np.abs(Wr[:3] - np.einsum("cd,dmn->cmn", R, W[:3]))) < 1e-12 * scale
    assert np.max(np.abs(Wr[3] - W[3])) < 1e-12 * scale


def test_w_staged_equals_brute_force():
    w = wl.tiny_chain(n_atom=2, n_rad=6, n_ang=10, shells=(0, 1), n_mu=10, seed=4)
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    res = pivots.select(phi, dphi, w.grid_w, 10)
    xi, xit, _ = fit.fit(phi, dphi, res.pivots)
    for jas in (w.jastrow, wl.bh_jastrow(w.atoms, w.xyz, wl.bh_terms_c4(), np.random.default_rng(9), 0.2)):
        Wst, _ = wbuild.build(w.grid_xyz, w.grid_w, xi, xit, jas, batch=7)
        Wbf = wbuild.brute_force(w.grid_xyz, w.grid_w, xi, xit, jas)
        assert np.max(np.abs(Wst - Wbf)) < 1e-11 * np.max(np.abs(Wbf))


def test_stage1_bounded_values_and_bound():
    """stage1_bounded: its sums equal stage1's (pinned above through W against the
    brute-force double-grid sum) on ragged row batches, and its bound is fixed as
    sum_g' |w_g' xi_nu(g')| |K_c(g, g')| by four properties: one nonzero g' gives
    |calG| itself (a single term), the bound depends on |xi| only (sign flips),
    it adds over disjoint supports of xi, and it dominates |calG|."""
    w = wl.tiny_chain(n_atom=2, n_rad=6, n_ang=10, shells=(0, 1), n_mu=10, seed=4)
    rng = np.random.default_rng(17)
    n_g = w.grid_xyz.shape[0]
    rows = np.sort(rng.choice(n_g, 37, replace=False))
    xi = rng.standard_normal((5, n_g))
    for jas in (w.jastrow, wl.bh_jastrow(w.atoms, w.xyz, wl.bh_terms_c4(), np.random.default_rng(9), 0.2)):
        val, bnd = wbuild.stage1_bounded(w.grid_xyz, w.grid_w, xi, jas, rows, batch=8)
        ref = wbuild.stage1(w.grid_xyz, w.grid_w, xi, jas, g_rows=rows)
        assert np.max(np.abs(val - ref)) < 1e-13 * np.max(np.abs(ref))
        assert np.all(bnd >= np.abs(val) * (1 - 1e-14))
        assert np.any(bnd > 1.5 * np.abs(val))          # mixed signs do cancel
        flip = xi * rng.choice([-1.0, 1.0], xi.shape)
        _, bflip = wbuild.stage1_bounded(w.grid_xyz, w.grid_w, flip, jas, rows, batch=8)
        assert np.max(np.abs(bflip - bnd)) < 1e-13 * np.max(bnd)
        mask = rng.random(n_g) < 0.5
        _, b1 = wbuild.stage1_bounded(w.grid_xyz, w.grid_w, xi * mask, jas, rows, batch=8)
        _, b2 = wbuild.stage1_bounded(w.grid_xyz, w.grid_w, xi * ~mask, jas, rows, batch=8)
        assert np.max(np.abs(b1 + b2 - bnd)) < 1e-13 * np.max(bnd)
        one = np.zeros_like(xi)
        one[:, 3] = xi[:, 3]
        v1, b1 = wbuild.stage1_bounded(w.grid_xyz, w.grid_w, one, jas, rows, batch=8)
        assert np.array_equal(b1, np.abs(v1))

def test_zero_jastrow_gives_zero(h6):
    w, phi, dphi = h6
    res = pivots.select(phi, dphi, w.grid_w, 24)
    xi, xit, _ = fit.fit(phi, dphi, res.pivots)
    jas = wl.radial_jastrow(w.xyz)
    jas.cusp = False
    W, calG = wbuild.build(w.grid_xyz, w.grid_w, xi, xit, jas)
    assert np.all(W == 0.0) and np.all(calG == 0.0)


def test_radial_u3_symmetric_and_coulomb_like(tiny):
    """Radial Jastrow: |grad u|^2 = u'(r)^2 is symmetric, so u3 is symmetric,
    and at full scalar rank K3^{pq}_{rs} equals the direct double-grid
    integral (pr|u'^2|qs)."""
    w, phi, dphi = tiny
    n = w.n_orb
    res = pivots.select(phi, dphi, w.grid_w, n * (n + 1) // 2, mode="scalar")
    P = res.piv_s
    xi, _, _ = fit.fit(phi, dphi, P, channels=(0,))
    calG = wbuild.stage1(w.grid_xyz, w.grid_w, xi, w.jastrow)
    u3 = (xi * w.grid_w) @ calG[3].T
    assert np.max(np.abs(u3 - u3.T)) < 1e-10 * np.max(np.abs(u3))
    # direct: sum_{g,g'} w w phi_p phi_r (g) u'(r)^2 phi_q phi_s (g')
    dv = w.grid_xyz[:, None, :] - w.grid_xyz[None, :, :]
    r = np.sqrt(np.sum(dv * dv, axis=2))
    k = 1.0 / (4.0 * (1.0 + r) ** 4)
    np.fill_diagonal(k, 0.0)
    C = phi[:, P]
    for (p, rr, q, s) in [(0, 0, 1, 1), (0, 1, 2, 2), (1, 2, 0, 2), (2, 2, 2, 2)]:
        direct = (w.grid_w * phi[p] * phi[rr]) @ k @ (w.grid_w * phi[q] * phi[s])
        isdf = (C[p] * C[rr]) @ u3 @ (C[q] * C[s])
        assert abs(isdf - direct) < 1e-8 * abs(direct)


# ---------------------------------------------------------------- xTC

def _pre_isdf_du(w, phi, n_occ, jas):
    """Delta U of Eqs. deltaU-four / deltaU-fields / deltaU-preisdf, by
    direct grid sums (no ISDF)."""
    n, n_g = phi.shape
    gw = w.grid_w
    K = jastrow.kernels(w.grid_xyz, w.grid_xyz, jas, np.arange(n_g), np.arange(n_g))[:3]
    gamma = np.zeros((n, n))
    gamma[np.arange(n_occ), np.arange(n_occ)] = 1.0
    rho = phi[:, None, :] * phi[None, :, :]                       # [a, b, g]
    rho_g = np.einsum("tu,tug->g", gamma, rho)
    beta = np.einsum("ut,tsg->usg", gamma, rho)
    A = np.einsum("abh,cgh->abgc", rho * gw, K)                   # sum_g' w rho K(g,g')
    Ag = np.einsum("h,cgh->gc", rho_g * gw, K)
    B = np.einsum("ush,cgh->usgc", beta * gw, K)
    T1 = 2 * np.einsum("g,prg,gc,qsgc->pqrs", gw, rho, Ag, A)
    T2 = -np.einsum("g,prg,usgc,qugc->pqrs", gw, rho, B, A)
    T3 = -np.einsum("g,prgc,usg,qugc->pqrs", gw, A, beta, A) \
         - np.einsum("g,prgc,usgc,qug->pqrs", gw, A, B, rho)
    T4 = np.einsum("g,g,prgc,qsgc->pqrs", gw, rho_g, A, A)
    T = T1 + T2 + T3 + T4
    return -(T + np.transpose(T, (1, 0, 3, 2)))


def test_xtc_full_rank_equals_pre_isdf(tiny):
    w, phi, dphi = tiny
    n = w.n_orb
    res = pivots.select(phi, dphi, w.grid_w, n * (n + 1) // 2, mode="scalar")
    P = res.piv_s
    xi, _, _ = fit.fit(phi, dphi, P, channels=(0,))
    calG = wbuild.stage1(w.grid_xyz, w.grid_w, xi, w.jastrow)
    phiP = xtc.pivot_factors(phi, P)
    n_occ = 1
    _, _, D = xtc.d_kernels(w.grid_w, xi, calG, xtc.g_nu(phiP, n_occ))
    X = xtc.x_projector(w.grid_w, xi, calG, phiP, n_occ)
    idx = np.arange(n)
    dU = energies.du_tensor(D, X, phiP, idx)
    ref = _pre_isdf_du(w, phi, n_occ, w.jastrow)
    assert np.max(np.abs(dU - ref)) < 1e-7 * np.max(np.abs(ref))


def _three_body_L(grid, gw, phi, jas):
    """L^{pqr}_{stu} of Eq. Hbar-2nd, index order [p, q, r, s, t, u]: the
    three-body operator of the BCH expansion (Eq. Hbar-bch), the sum over the
    centre electron a of grad_a u(a,b) . grad_a u(a,c) with each centre counted
    once, against phi_p phi_s (1), phi_q phi_t (2), phi_r phi_u (3).  The triple
    grid sum runs through F^a_b(g) = sum_g' w_g' phi_a phi_b (g') grad u(g, g'),
    an exact refactoring of it (see test_three_body_fields_equal_triple_sum)."""
    n_g = grid.shape[0]
    K = jastrow.kernels(grid, grid, jas, np.arange(n_g), np.arange(n_g))[:3]
    rho = phi[:, None, :] * phi[None, :, :]
    F = np.einsum("abh,cgh->abgc", rho * gw, K)
    return (np.einsum("g,psg,qtgc,rugc->pqrstu", gw, rho, F, F)
            + np.einsum("g,qtg,psgc,rugc->pqrstu", gw, rho, F, F)
            + np.einsum("g,rug,psgc,qtgc->pqrstu", gw, rho, F, F))


def _normal_ordered_du(L, n_occ):
    """Normal ordering the three-body part -1/6 L a+a+a+aaa of Eq. Hbar-2nd
    against the closed-shell determinant leaves the two-body operator
    -1/2 v a+_p a+_q a_s a_r with
        v^{pq}_{rs} = sum_{k occ} [2 L^{pqk}_{rsk} - L^{pqk}_{ksr} - L^{pqk}_{rks}]
    (the third electron contracted directly, summed over both spins, minus its
    exchange with electron 1 or 2, same spin only).  Eq. xtc-hamiltonian
    carries the two-body part as +1/2 DeltaU, so DeltaU = -v."""
    v = np.zeros(L.shape[:2] + L.shape[3:5])
    for k in range(n_occ):
        v += 2.0 * L[:, :, k, :, :, k]
        v -= np.transpose(L[:, :, k, k, :, :], (0, 1, 3, 2))
        v -= L[:, :, k, :, k, :]
    return -v


def test_three_body_fields_equal_triple_sum():
    """The field refactoring of L against the literal triple sum over grid
    points (g1, g2, g3) on a 48-point grid."""
    w = wl.tiny_chain(n_atom=2, n_rad=4, n_ang=6, shells=(0,), seed=5)
    jas = wl.bh_jastrow(w.atoms, w.xyz, wl.bh_terms_c4(), np.random.default_rng(4), 0.2)
    phi, _ = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    n_g = w.n_g
    K = jastrow.kernels(w.grid_xyz, w.grid_xyz, jas, np.arange(n_g), np.arange(n_g))[:3]
    O = np.einsum("xab,xac->abc", K, K)               # grad_a u(a,b) . grad_a u(a,c)
    G = O + np.transpose(O, (1, 0, 2)) + np.transpose(O, (1, 2, 0))
    rho = phi[:, None, :] * phi[None, :, :] * w.grid_w
    L_sum = np.einsum("psa,qtb,ruc,abc->pqrstu", rho, rho, rho, G)
    L = _three_body_L(w.grid_xyz, w.grid_w, phi, jas)
    assert np.max(np.abs(L - L_sum)) < 1e-12 * np.max(np.abs(L_sum))


def test_xtc_equals_normal_ordered_three_body_term():
    """Delta U of Eqs. deltaU-four .. deltaU-preisdf, and the oracle's ISDF
    route at full scalar rank, against the normal-ordered three-body
    operator L of Eq. Hbar-2nd (4 orbitals, 2 occupied; radial and
    two-type multi-centre correlators).  Pins the signs and factors of
    Terms 1-4 and the reading that L counts each centre electron once."""
    w = wl.tiny_chain(n_atom=4, n_rad=12, n_ang=20, shells=(0,), n_mu=10, seed=11)
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    n, n_occ = w.n_orb, w.n_occ
    assert (n, n_occ) == (4, 2)
    res = pivots.select(phi, dphi, w.grid_w, n * (n + 1) // 2, mode="scalar")
    P = res.piv_s
    xi, _, _ = fit.fit(phi, dphi, P, channels=(0,))
    phiP = xtc.pivot_factors(phi, P)
    bh = wl.bh_jastrow(w.atoms, w.xyz, wl.bh_terms_c4(), np.random.default_rng(9), 0.2)
    for jas in (w.jastrow, bh):
        ref = _normal_ordered_du(_three_body_L(w.grid_xyz, w.grid_w, phi, jas), n_occ)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(_pre_isdf_du(w, phi, n_occ, jas) - ref)) < 1e-12 * scale
        calG = wbuild.stage1(w.grid_xyz, w.grid_w, xi, jas)
        _, _, D = xtc.d_kernels(w.grid_w, xi, calG, xtc.g_nu(phiP, n_occ))
        X = xtc.x_projector(w.grid_w, xi, calG, phiP, n_occ)
        dU = energies.du_tensor(D, X, phiP, np.arange(n))
        assert np.max(np.abs(dU - ref)) < 1e-7 * scale


def _normal_ordered_scalars(L, n_occ):
    """One-body increment and constant of the plain-form Hamiltonian from
    normal ordering -1/6 L (Eq. Hbar-2nd) against the closed-shell determinant.

    The doubly and triply contracted parts take the three-electron
    antisymmetrizer A3 = 1 - P12 - P13 - P23 + two 3-cycles, summed over the
    spins the contracted orbitals may carry (each permutation term gets the
    count of spin assignments it allows):
      f_pq = -1/2 sum_{kl} [4 L^{pkl}_{qkl} - 2 L^{pkl}_{kql} - 2 L^{pkl}_{lkq}
                            - 2 L^{pkl}_{qlk} + L^{pkl}_{klq} + L^{pkl}_{lqk}]
      c    = -1/6 sum_{klm} [8 L^{klm}_{klm} - 4 (L^{klm}_{lkm} + L^{klm}_{mlk} + L^{klm}_{kml})
                             + 2 (L^{klm}_{lmk} + L^{klm}_{mkl})]
    Rewriting the normal-ordered two-body part 1/2 DeltaU {a+a+aa} in plain
    form adds -sum_k (2 DeltaU^{pk}_{qk} - DeltaU^{pk}_{kq}) to the one-body
    term and +E_dU to the constant, and rewriting the normal-ordered one-body
    part adds -E_dU, so the constant is c alone.  Returns (Delta h [n][n], E0)."""
    occ = range(n_occ)
    dU = _normal_ordered_du(L, n_occ)
    f = np.zeros(L.shape[:1] * 2)
    for a in occ:
        for b in occ:
            f += (4 * L[:, a, b, :, a, b] - 2 * L[:, a, b, a, :, b] - 2 * L[:, a, b, b, a, :]
                  - 2 * L[:, a, b, :, b, a] + L[:, a, b, a, b, :] + L[:, a, b, b, :, a])
    f *= -0.5
    conv = -sum(2 * dU[:, k, :, k] - dU[:, k, k, :] for k in occ)
    c = 0.0
    for k in occ:
        for l in occ:
            for m in occ:
                c += (8 * L[k, l, m, k, l, m]
                      - 4 * (L[k, l, m, l, k, m] + L[k, l, m, m, l, k] + L[k, l, m, k, m, l])
                      + 2 * (L[k, l, m, l, m, k] + L[k, l, m, m, k, l]))
    return f + conv, -c / 6.0


def test_delta_h_and_e0_equal_normal_ordered_three_body_term():
    """Eqs. xtc-deltah and xtc-const (Delta h from a partial contraction of
    DeltaU, E0 = -2/3 sum_i Delta h_ii) against the one-body part and the
    constant of the normal-ordered three-body operator L, through the
    oracle's energies at full scalar rank (4 orbitals, 2 occupied)."""
    w = wl.tiny_chain(n_atom=4, n_rad=12, n_ang=20, shells=(0,), n_mu=10, seed=11)
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    n, n_occ = w.n_orb, w.n_occ
    res = pivots.select(phi, dphi, w.grid_w, n * (n + 1) // 2, mode="scalar")
    P = res.piv_s
    xi, _, _ = fit.fit(phi, dphi, P, channels=(0,))
    phiP = xtc.pivot_factors(phi, P)
    dphiP = [dphi[c][:, P].T for c in range(3)]
    bh = wl.bh_jastrow(w.atoms, w.xyz, wl.bh_terms_c4(), np.random.default_rng(9), 0.2)
    for jas in (w.jastrow, bh):
        dh_ref, E0_ref = _normal_ordered_scalars(_three_body_L(w.grid_xyz, w.grid_w, phi, jas),
                                                 n_occ)
        calG = wbuild.stage1(w.grid_xyz, w.grid_w, xi, jas)
        _, _, D = xtc.d_kernels(w.grid_w, xi, calG, xtc.g_nu(phiP, n_occ))
        X = xtc.x_projector(w.grid_w, xi, calG, phiP, n_occ)
        occ = np.arange(n_occ)
        dh = energies.delta_h_occ(energies.du_tensor(D, X, phiP, occ))
        assert np.max(np.abs(dh - np.diag(dh_ref)[:n_occ])) < 1e-7 * np.max(np.abs(dh_ref))
        E = energies.energies(np.zeros((4, len(P), len(P))), D, X, phiP, dphiP, n_occ)
        assert abs(E["E0"] - E0_ref) < 1e-7 * abs(E0_ref)


def test_projector_equals_dense_and_symmetry(h6):
    w, phi, dphi = h6
    res = pivots.select(phi, dphi, w.grid_w, 30)
    xi, xit, _ = fit.fit(phi, dphi, res.pivots)
    calG = wbuild.stage1(w.grid_xyz, w.grid_w, xi, w.jastrow)
    phiP = xtc.pivot_factors(phi, res.pivots)
    phiP = phiP[:, :8]
    X2, X3 = xtc.x_dense(w.grid_w, xi, calG, phiP, w.n_occ)
    Xp = xtc.x_projector(w.grid_w, xi, calG, phiP, w.n_occ)
    ref = X2 + X3
    assert np.linalg.norm(Xp - ref) < 1e-10 * np.linalg.norm(ref)
    assert np.max(np.abs(Xp - np.transpose(Xp, (1, 0, 2)))) < 1e-12 * np.max(np.abs(Xp))
    D4, D1, _ = xtc.d_kernels(w.grid_w, xi, calG, xtc.g_nu(phiP, w.n_occ))
    assert np.max(np.abs(D4 - D4.T)) < 1e-12 * np.max(np.abs(D4))


def test_particle_exchange(h6):
    w, phi, dphi = h6
    res = pivots.select(phi, dphi, w.grid_w, 30)
    xi, xit, _ = fit.fit(phi, dphi, res.pivots)
    W, calG = wbuild.build(w.grid_xyz, w.grid_w, xi, xit, w.jastrow)
    phiP = xtc.pivot_factors(phi, res.pivots)
    dphiP = [dphi[c][:, res.pivots].T for c in range(3)]
    idx = np.arange(5)
    K = energies.k_tensor(W, phiP, dphiP, idx)
    assert np.max(np.abs(K - np.transpose(K, (1, 0, 3, 2)))) < 1e-12 * np.max(np.abs(K))
    # K is not Hermitian in the pair-block sense (Sec. IV.A)
    assert np.max(np.abs(K - np.transpose(K, (2, 3, 0, 1)))) > 1e-6 * np.max(np.abs(K))


def test_k_tensor_full_rank_equals_direct_double_grid_sum(tiny):
    """At full fused rank (both channels' product spaces spanned) the ISDF
    four-index K of Eq. K-recombine-final equals its pre-ISDF definition,
    K1^{pq}_{rs} = sum_c sum_{g,g'} w w phi_p d_c phi_r (g) K_c(g,g') phi_q phi_s (g'),
    K3 with K_sq and rho_pr rho_qs, combined as 1/2 P12 [K1 - K1swap + K3]."""
    w, phi, dphi = tiny
    n, n_g = phi.shape
    res = pivots.select(phi, dphi, w.grid_w, 33)
    assert res.rank_exhausted and len(res.pivots) == 30  # 6 scalar + 27 gradient, 3 shared
    P = res.pivots
    xi, xit, _ = fit.fit(phi, dphi, P)
    W, _ = wbuild.build(w.grid_xyz, w.grid_w, xi, xit, w.jastrow)
    phiP = xtc.pivot_factors(phi, P)
    dphiP = [dphi[c][:, P].T for c in range(3)]
    K = energies.k_tensor(W, phiP, dphiP, np.arange(n))
    Kc = jastrow.kernels(w.grid_xyz, w.grid_xyz, w.jastrow, np.arange(n_g), np.arange(n_g))
    gw = w.grid_w
    rho = phi[:, None, :] * phi[None, :, :]
    K1 = np.zeros((n,) * 4)
    for c in range(3):
        grad_pr = gw * phi[:, None, :] * dphi[c][None, :, :]
        K1 += np.einsum("prg,gh,qsh->pqrs", grad_pr, Kc[c], gw * rho)
    K3 = np.einsum("prg,gh,qsh->pqrs", gw * rho, Kc[3], gw * rho)
    T = K1 - np.transpose(K1, (2, 3, 0, 1)) + K3
    direct = 0.5 * (T + np.transpose(T, (1, 0, 3, 2)))
    assert np.max(np.abs(K - direct)) < 1e-9 * np.max(np.abs(direct))


def test_e0_is_a_third_of_e_du(h6):
    """With Eqs. xtc-deltah and xtc-const, sum_i Delta h_ii = -E_dU / 2, so
    E0 = E_dU / 3 exactly (an index swap in Delta h breaks it)."""
    w, phi, dphi = h6
    res = pivots.select(phi, dphi, w.grid_w, 40)
    xi, xit, _ = fit.fit(phi, dphi, res.pivots)
    W, calG = wbuild.build(w.grid_xyz, w.grid_w, xi, xit, w.jastrow)
    phiP = xtc.pivot_factors(phi, res.pivots)
    dphiP = [dphi[c][:, res.pivots].T for c in range(3)]
    _, _, D = xtc.d_kernels(w.grid_w, xi, calG, xtc.g_nu(phiP, w.n_occ))
    X = xtc.x_projector(w.grid_w, xi, calG, phiP, w.n_occ)
    E = energies.energies(W, D, X, phiP, dphiP, w.n_occ)
    assert abs(E["E0"] - E["E_dU"] / 3.0) < 1e-12 * abs(E["E_dU"])


# ---------------------------------------------------------------- adjoint

def test_dgrad_dtheta_matches_fd():
    from oracle import adjoint
    atoms, xyz = wl.h_chain(3, 1.8)
    jas = wl.bh_jastrow(atoms, xyz, wl.bh_terms_c4(), np.random.default_rng(4), scale=0.3)
    jas.b = np.array([1.2])
    jas.d = 0.9
    rng = np.random.default_rng(8)
    ri = rng.normal(size=(5, 3)) * 2
    rj = rng.normal(size=(4, 3)) * 2
    an = adjoint.dgrad_dtheta(ri, rj, jas)
    th = adjoint.get_theta(jas)
    h = 1e-6
    for p in range(len(th)):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (jastrow.grad1_u(ri, rj, adjoint.set_theta(jas, tp))
              - jastrow.grad1_u(ri, rj, adjoint.set_theta(jas, tm))) / (2 * h)
        assert np.max(np.abs(fd - an[p])) < 1e-7 * max(1.0, np.max(np.abs(an[p]))), p


def test_adjoint_gradient_matches_fd_of_loss():
    """dL/dtheta of L = sum_c <Wbar^c, W^c> against central differences."""
    from oracle import adjoint
    w = wl.tiny_chain(n_atom=2, n_rad=6, n_ang=10, shells=(0, 1), n_mu=8, seed=6,
                      jkind="bh", jterms=wl.bh_terms_c4()[:9])
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    res = pivots.select(phi, dphi, w.grid_w, w.n_mu)
    xi, xit, _ = fit.fit(phi, dphi, res.pivots)
    Wbar = wl.seeded_matrix((4, w.n_mu, w.n_mu), 99)
    jas = w.jastrow
    jas.coef = jas.coef * 4.0
    g = adjoint.grad(w.grid_xyz, w.grid_w, xi, xit, jas, Wbar, batch=37)
    th = adjoint.get_theta(jas)
    h = 1e-5
    for p in range(len(th)):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (adjoint.loss(w.grid_xyz, w.grid_w, xi, xit, adjoint.set_theta(jas, tp), Wbar)
              - adjoint.loss(w.grid_xyz, w.grid_w, xi, xit, adjoint.set_theta(jas, tm), Wbar)) / (2 * h)
        assert abs(fd - g[p]) < 1e-6 * max(1.0, abs(g[p])), (p, fd, g[p])


def test_adjoint_with_chi_matches_fd_of_loss():
    """The adjoint with the one-body term present: chi carries no parameter of
    theta, but it enters K_c and so the M^sq K_c factor of the gradient."""
    from oracle import adjoint
    w = wl.tiny_chain(n_atom=2, n_rad=5, n_ang=8, shells=(0, 1), n_mu=6, seed=3,
                      jkind="bh", jterms=wl.bh_terms_c4()[:5])
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    res = pivots.select(phi, dphi, w.grid_w, w.n_mu)
    xi, xit, _ = fit.fit(phi, dphi, res.pivots)
    Wbar = wl.seeded_matrix((4, w.n_mu, w.n_mu), 5)
    jas = wl.with_chi(w.jastrow, [1.0], 2 * w.n_occ, beta=1.1)
    jas.coef = jas.coef * 4.0
    g = adjoint.grad(w.grid_xyz, w.grid_w, xi, xit, jas, Wbar, batch=29)
    th = adjoint.get_theta(jas)
    h = 1e-5
    for p in range(len(th)):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (adjoint.loss(w.grid_xyz, w.grid_w, xi, xit, adjoint.set_theta(jas, tp), Wbar)
              - adjoint.loss(w.grid_xyz, w.grid_w, xi, xit, adjoint.set_theta(jas, tm), Wbar)) / (2 * h)
        assert abs(fd - g[p]) < 1e-6 * max(1.0, abs(g[p])), (p, fd, g[p])


def test_adjoint_linear_in_seed():
    from oracle import adjoint
    w = wl.tiny_chain(n_atom=2, n_rad=5, n_ang=8, shells=(0,), n_mu=3, seed=2,
                      jkind="bh", jterms=wl.BH_TERMS_C3[:4])
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    res = pivots.select(phi, dphi, w.grid_w, w.n_mu)
    xi, xit, _ = fit.fit(phi, dphi, res.pivots)
    A = wl.seeded_matrix((4, 3, 3), 1)
    B = wl.seeded_matrix((4, 3, 3), 2)
    gA = adjoint.grad(w.grid_xyz, w.grid_w, xi, xit, w.jastrow, A)
    gB = adjoint.grad(w.grid_xyz, w.grid_w, xi, xit, w.jastrow, B)
    gAB = adjoint.grad(w.grid_xyz, w.grid_w, xi, xit, w.jastrow, 2.0 * A - 3.0 * B)
    assert np.allclose(gAB, 2.0 * gA - 3.0 * gB, rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------- learned proposer

def test_mlp_gradient_matches_fd():
    from oracle import mlp
    rng = np.random.default_rng(0)
    x = rng.standard_normal((40, mlp.F))
    y = (rng.random(40) < 0.2).astype(float)
    th = mlp.init_params(1) + 0.01 * rng.standard_normal(mlp.N_PARAMS)
    l, g = mlp.loss_and_grad(th, x, y, 4.0, rounding=False)
    h = 1e-6
    for p in rng.choice(mlp.N_PARAMS, 25, replace=False).tolist() + [mlp.N_PARAMS - 1]:
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (mlp.loss_and_grad(tp, x, y, 4.0, False)[0] - mlp.loss_and_grad(tm, x, y, 4.0, False)[0]) / (2 * h)
        assert abs(fd - g[p]) < 1e-7 * max(1.0, abs(g[p])), (p, fd, g[p])


def test_mlp_bce_at_zero_logit_and_bf16_rounding():
    from oracle import mlp
    th = np.zeros(mlp.N_PARAMS)
    x = np.ones((10, mlp.F))
    y = np.array([1.0, 0, 0, 1, 0, 0, 0, 0, 0, 0])
    l, _ = mlp.loss_and_grad(th, x, y, 3.0)
    # softplus(0) = log 2 for every point, weighted by 3 for the two positives
    assert abs(l - math.log(2.0) * (3.0 * 2 + 8) / 10) < 1e-15
    # bf16 rounding: exactly representable values are fixed points, ties go to even
    vals = np.array([1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-30])
    r = mlp.bf16_round(vals)
    assert r[0] == 1.0 and r[1] == 1.0 + 2 ** -7
    assert r[2] == 1.0                    # halfway, rounds to the even neighbour 1.0
    assert r[3] == 1.0 + 2 ** -6          # halfway, rounds to the even neighbour
    assert r[4] == -2.5
    assert abs(r[5] - 3.0e-30) < 3.0e-30 * 2 ** -8


def test_adam_first_step_is_sign_step():
    from oracle import mlp
    th = np.array([0.5, -1.0, 2.0])
    g = np.array([3.0, -0.2, 1e-3])
    new, m, v = mlp.adam(th, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first moments equal g and g^2: the step is lr * g / (|g| + eps)
    assert np.allclose(new, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_candidates_and_fit_error():
    from oracle import mlp
    s = np.array([0.5, 2.0, 2.0, -1.0, 0.7, 2.0, 0.1])
    assert mlp.candidates(s, 2).tolist() == [1, 2]      # ties by lowest index
    assert mlp.candidates(s, 4).tolist() == [1, 2, 4, 5]
    # at full scalar rank the fit error vanishes
    w = wl.tiny_chain(n_atom=3, n_rad=16, n_ang=26, shells=(0,), seed=11)
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    res = pivots.select(phi, dphi, w.grid_w, 6, mode="scalar")
    assert mlp.fit_error(phi, w.grid_w, res.piv_s) < 1e-12
    res3 = pivots.select(phi, dphi, w.grid_w, 3, mode="scalar")
    e3 = mlp.fit_error(phi, w.grid_w, res3.piv_s)
    assert 0 < e3 < 1


def test_features_carry_the_pivot_diagonals(h6):
    """Features 0 and 1 are monotone in the scalar and gradient pivot
    diagonals d^(0) of Alg. 1 (Sec. II.D), so their argmax is each channel's
    first pivot; features 5 and 6 are the sorted nearest-nucleus distances."""
    from oracle import mlp
    w, phi, dphi = h6
    f = mlp.features(phi, dphi, w.grid_w, w.grid_xyz, w.xyz)
    assert f.shape == (w.n_g, 8) and np.all(np.isfinite(f))
    first_s = pivots.select(phi, dphi, w.grid_w, 1, mode="scalar").piv_s[0]
    first_v = pivots.select(phi, dphi, w.grid_w, 1, mode="gradient").piv_v[0]
    assert int(np.argmax(f[:, 0])) == first_s
    assert int(np.argmax(f[:, 1])) == first_v
    assert np.all(f[:, 5] <= f[:, 6])
    d = np.linalg.norm(w.grid_xyz[:, None, :] - w.xyz[None, :, :], axis=2)
    assert np.allclose(f[:, 5], d.min(axis=1) / 5.0, rtol=0, atol=1e-15)


def test_delta_h_all_orbitals_equals_normal_ordered_three_body_term():
    """Eq. xtc-deltah over every (p, q), not only the occupied diagonal, from
    the full four-index DeltaU at full scalar rank, against the one-body part
    of the normal-ordered three-body operator (4 orbitals, 2 occupied)."""
    w = wl.tiny_chain(n_atom=4, n_rad=12, n_ang=20, shells=(0,), n_mu=10, seed=11)
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    n, n_occ = w.n_orb, w.n_occ
    res = pivots.select(phi, dphi, w.grid_w, n * (n + 1) // 2, mode="scalar")
    P = res.piv_s
    xi, _, _ = fit.fit(phi, dphi, P, channels=(0,))
    phiP = xtc.pivot_factors(phi, P)
    occ = np.arange(n_occ)
    bh = wl.bh_jastrow(w.atoms, w.xyz, wl.bh_terms_c4(), np.random.default_rng(9), 0.2)
    for jas in (w.jastrow, bh):
        dh_ref, E0_ref = _normal_ordered_scalars(_three_body_L(w.grid_xyz, w.grid_w, phi, jas),
                                                 n_occ)
        calG = wbuild.stage1(w.grid_xyz, w.grid_w, xi, jas)
        _, _, D = xtc.d_kernels(w.grid_w, xi, calG, xtc.g_nu(phiP, n_occ))
        X = xtc.x_projector(w.grid_w, xi, calG, phiP, n_occ)
        dU = energies.du_tensor(D, X, phiP, np.arange(n))
        dh = energies.delta_h(dU, occ)
        assert np.max(np.abs(dh - dh_ref)) < 1e-7 * np.max(np.abs(dh_ref))
        assert abs(energies.e0_xtc(dh, occ) - E0_ref) < 1e-7 * abs(E0_ref)


def test_fock_closed_form_for_separable_two_body():
    """Eq. xtc-fock on a two-body correction of product form
    W^{pq}_{rs} = u_p u_r v_q v_s (K = -W, DeltaU = 0): the Coulomb sum is
    sum_i W^{pi}_{qi} = u_p u_q sum_i v_i^2 and the exchange sum is
    sum_i W^{pi}_{iq} = u_p v_q sum_i u_i v_i, so
    f_pq = 2 u_p u_q S_vv - u_p v_q S_uv (worked by hand; a Coulomb or
    exchange index in the wrong slot gives another matrix)."""
    rng = np.random.default_rng(12)
    n, occ = 5, np.arange(2)
    u, v = rng.standard_normal(n), rng.standard_normal(n)
    Wt = np.einsum("p,r,q,s->pqrs", u, u, v, v)
    f = energies.fock_xtc(-Wt, np.zeros_like(Wt), occ)
    Svv, Suv = float(np.sum(v[occ] ** 2)), float(np.sum(u[occ] * v[occ]))
    assert np.max(np.abs(f - (2.0 * np.outer(u, u) * Svv - np.outer(u, v) * Suv))) < 1e-14


def test_fock_trace_matches_closed_shell_energies(h6):
    """sum_i f^xTC_ii = sum_i Delta h_ii - E_K + E_dU = E_dU / 2 - E_K on the
    occupied block (Eq. xtc-fock traced against the closed-shell functionals)."""
    w, phi, dphi = h6
    res = pivots.select(phi, dphi, w.grid_w, 30)
    xi, xit, _ = fit.fit(phi, dphi, res.pivots)
    W, calG = wbuild.build(w.grid_xyz, w.grid_w, xi, xit, w.jastrow)
    phiP = xtc.pivot_factors(phi, res.pivots)
    dphiP = [dphi[c][:, res.pivots].T for c in range(3)]
    _, _, D = xtc.d_kernels(w.grid_w, xi, calG, xtc.g_nu(phiP, w.n_occ))
    X = xtc.x_projector(w.grid_w, xi, calG, phiP, w.n_occ)
    idx = np.arange(6)
    occ = np.arange(w.n_occ)
    K = energies.k_tensor(W, phiP, dphiP, idx)
    dU = energies.du_tensor(D, X, phiP, idx)
    f = energies.fock_xtc(K, dU, occ)
    E = energies.energies(W, D, X, phiP, dphiP, w.n_occ)
    tr = float(np.trace(f[np.ix_(occ, occ)]))
    assert abs(tr - (E["E_dU"] / 2.0 - E["E_K"])) < 1e-12 * (abs(E["E_K"]) + abs(E["E_dU"]))
