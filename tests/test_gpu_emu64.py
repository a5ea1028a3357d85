"""FP64 products emulated on the tensor cores (isdf_dgemm_emulated) and the
fit that uses them (isdf_fit with fit_mode 1), against extended-precision
products, exact integer products and the FP64 oracle of the fit (Sec. II.D's
normal equations, Sec. IV.B's solves)."""
import numpy as np
import pytest
import torch

from synth import workloads as wl
from oracle import orbitals, pivots, fit

pytestmark = pytest.mark.gpu

EPS = np.finfo(float).eps


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_17314_b300 import build
    build.build()
    from paper_2607_17314_b300 import api
    return api


def cu(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dt).cuda()


def host(t):
    return t.detach().cpu().numpy()


def exact_product(A, B):
    """A B in extended precision (64-bit significand), then rounded to FP64."""
    return (A.astype(np.longdouble) @ B.astype(np.longdouble)).astype(np.float64)


def pow2_above(x):
    """2^e with e the smallest integer such that x < 2^e (0 where x = 0): the
    power-of-two scale the emulation takes for a row or column maximum."""
    x = np.asarray(x, dtype=float)
    out = np.zeros_like(x)
    nz = x > 0
    out[nz] = 2.0 ** (np.floor(np.log2(x[nz])) + 1.0)
    return out


def scale_bound(A, B):
    """(K + 4) 2^-52 2^(e_m + e_n), the emulation's per-element error bound
    (2^e_m > max_k|A_mk|, 2^e_n > max_k|B_kn|): the dropped digit pairs give at
    most ~2^-53.2 of the scale per term, the truncated digits 2^-55, and the
    lowest level pair's rounding in the 64-bit combination 1 unit of 2^-52."""
    K = A.shape[1]
    return (K + 4) * 2.0 ** -52 * pow2_above(np.abs(A).max(1))[:, None] * \
        pow2_above(np.abs(B).max(0))[None, :]


@pytest.mark.parametrize("M,N,K,spread", [(300, 130, 128, 0.0), (129, 65, 37, 3.0),
                                          (200, 257, 300, 6.0), (7, 3, 1, 0.0),
                                          (150, 70, 1100, 2.0)])
def test_emulated_product_within_bound(api, M, N, K, spread):
    """Ragged M, N (not multiples of the 128 x 64 tiles); K within one
    tensor-core run, K over three runs summed in 64-bit integers in one work
    unit, and K = 1100 (nine runs) split over work units added with FP64
    atomics; rows and columns of wide dynamic range, a zero row, a zero column
    and mixed signs."""
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-spread, spread, (M, K))
    B = rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-spread, spread, (K, N))
    A[min(2, M - 1)] = 0.0
    B[:, min(1, N - 1)] = 0.0
    C = host(api.isdf_dgemm_emulated(cu(A), cu(B)))
    ref = exact_product(A, B)
    err = np.abs(C - ref)
    bound = scale_bound(A, B)
    ratio = float(np.max(err / np.where(bound > 0, bound, 1.0)))
    fp64 = float(np.max(np.abs(A @ B - ref) / np.where(bound > 0, bound, 1.0)))
    print(f"M={M} N={N} K={K}: error / bound {ratio:.3e} (FP64 GEMM {fp64:.3e})")
    assert np.all(err <= bound), ratio
    assert np.all(C[min(2, M - 1)] == 0.0) and np.all(C[:, min(1, N - 1)] == 0.0)


def test_emulated_product_of_integers_is_exact(api):
    """Integer matrices whose FP64 product is exact: every digit product and
    level sum is an integer, so the emulated result is bit-identical."""
    rng = np.random.default_rng(3)
    A = rng.integers(-120, 121, (150, 300)).astype(float)
    B = rng.integers(-120, 121, (300, 70)).astype(float)
    C = host(api.isdf_dgemm_emulated(cu(A), cu(B)))
    assert np.array_equal(C, A @ B)


def test_emulated_product_accumulates(api):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((70, 90))
    B = rng.standard_normal((90, 40))
    C0 = rng.standard_normal((70, 40))
    out = cu(C0)
    api.isdf_dgemm_emulated(cu(A), cu(B), alpha=-1.5, out=out)
    ref = (C0.astype(np.longdouble) - 1.5 * (A.astype(np.longdouble) @ B.astype(np.longdouble))
           ).astype(np.float64)
    bound = 1.5 * scale_bound(A, B) + EPS * np.abs(C0)
    assert np.all(np.abs(host(out) - ref) <= bound)


def _fit_case(n_mu):
    w = wl.h6_chain()
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    res = pivots.select(phi, dphi, w.grid_w, n_mu)
    return w, phi, dphi, res.pivots


@pytest.mark.parametrize("n_mu", [96, 200])
def test_emulated_fit_against_oracle(api, n_mu):
    """Sec. II.D's normal equations solved with the emulated products (one
    block of 128 at N_mu = 96; two blocks, with trailing updates both ways,
    at N_mu = 200, where the scalar Gram's condition number is ~1e12): backward error at 1e-10 against the oracle's Grams and
    right-hand sides, forward agreement with the oracle within the Grams'
    condition number times 64 FP64 unit roundoffs (the emulated products carry
    about K 2^-52 of their scale, some 10x FP64's typical rounding)."""
    w, phi, dphi, piv = _fit_case(n_mu)
    xi, xig, jit = api.isdf_fit(cu(phi), cu(dphi), cu(piv, torch.int32), fit_mode=1)
    xo, xto, lams = fit.fit(phi, dphi, piv)
    assert np.allclose(jit, lams)
    Gm = fit.grams(phi, dphi, piv)
    Bm = fit.rhs(phi, dphi, piv)
    X = np.concatenate([host(xi)[None], host(xig)])
    Xo = np.concatenate([xo[None], xto])
    for c in range(4):
        G = Gm[c] + lams[c] * np.eye(Gm.shape[1])
        back = np.linalg.norm(G @ X[c] - Bm[c]) / (np.linalg.norm(G) * np.linalg.norm(X[c]))
        kappa = np.linalg.cond(G)
        fwd = np.linalg.norm(X[c] - Xo[c]) / np.linalg.norm(Xo[c])
        print(f"n_mu={n_mu} channel {c}: backward {back:.2e} cond {kappa:.2e} forward {fwd:.2e}")
        assert back < 1e-10, (c, back)
        assert fwd < max(1e-10, 64.0 * kappa * EPS), (c, fwd, kappa)


def test_emulated_fit_matches_fp64_fit_on_gpu(api):
    """fit_mode 1 against fit_mode 0 on the same GPU inputs (N_mu = 200)."""
    w, phi, dphi, piv = _fit_case(200)
    args = (cu(phi), cu(dphi), cu(piv, torch.int32))
    x1, g1, _ = api.isdf_fit(*args, fit_mode=1)
    x0, g0, _ = api.isdf_fit(*args, fit_mode=0)
    Gm = fit.grams(phi, dphi, piv)
    for c, (a, b) in enumerate([(x1, x0)] + [(g1[i], g0[i]) for i in range(3)]):
        kappa = np.linalg.cond(Gm[c])
        d = float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
        assert d < max(1e-10, 64.0 * kappa * EPS), (c, d, kappa)


def test_emulated_orbitals_within_bound(api):
    """Alg. 2 step 2 with the contractions C^T chi emulated (mode 1) against the
    same call with FP64 GEMMs (mode 0) on the H6 grid: both take the same basis
    values from the same kernel, so every value differs by at most the
    emulation's (n_bf + 4) 2^-52 2^(e_p + e_g) (2^e_p > max_f|C_fp|,
    2^e_g > max_f|chi_f(g)|) plus the FP64 GEMM's own rounding.  (Mode 0 against
    the oracle is the orbital parity test; there the two sides' exponentials
    differ by up to a r^2 units of FP64 rounding.)"""
    w = wl.h6_chain()
    b = w.basis
    args = (cu(b.center), cu(b.powers, torch.int32), cu(b.exps), cu(b.coefs), cu(w.mo_coef),
            cu(w.grid_xyz))
    phi1, dphi1 = api.isdf_eval_orbitals(*args, mode=1)
    phi0, dphi0 = api.isdf_eval_orbitals(*args, mode=0)
    v, g = orbitals.eval_ao(w.basis, w.grid_xyz)
    cmax = pow2_above(np.abs(w.mo_coef).max(0))[:, None]
    nbf = w.mo_coef.shape[0]
    csum = np.abs(w.mo_coef).T @ np.ones(nbf)
    planes = [(host(phi1), host(phi0), v)] + [(host(dphi1)[c], host(dphi0)[c], g[c]) for c in range(3)]
    for got, ref, ao in planes:
        amax = np.abs(ao).max(0)[None, :]
        # amax from the oracle's basis values: within a few units of a r^2 FP64 roundings
        # of the GPU's, hence the factor 2 on both scales
        bound = ((nbf + 4) * 2.0 ** -52 * cmax * pow2_above(2 * amax)
                 + (nbf + 8) * EPS * csum[:, None] * 2 * amax + 2.0 ** -1000)
        err = np.abs(got - ref)
        ratio = err / bound
        print("orbital error / bound", float(ratio.max()))
        assert np.all(ratio <= 1.0), float(ratio.max())
