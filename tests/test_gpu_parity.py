"""GPU parity of every step of the path against the FP64 oracle, through the
C ABI, on seeded inputs (H6 chain: 4800 points = 37.5 tiles of 128, N_mu = 96
< one 128 tile, and smaller ragged systems).

Tolerances: bit-exact pivot indices given identical inputs; 1e-10 relative
for FP64 paths (loosened only where the fit's conditioning amplifies FP64
rounding, stated per test); 1e-5 relative Frobenius per W channel and 1e-6 Ha
in the energies for the split-BF16 tensor-core path.
"""
import numpy as np
import pytest
import torch

from synth import workloads as wl
from oracle import orbitals, pivots, fit, wbuild, xtc, energies

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cu(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dt).cuda()


def host(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_17314_b300 import build
    build.build()
    import paper_2607_17314_b300 as P
    P._capi.load()
    return P


def oracle_case(w):
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    res = pivots.select(phi, dphi, w.grid_w, w.n_mu)
    xi, xit, lams = fit.fit(phi, dphi, res.pivots)
    W, calG = wbuild.build(w.grid_xyz, w.grid_w, xi, xit, w.jastrow)
    phiP = xtc.pivot_factors(phi, res.pivots)
    dphiP = [dphi[c][:, res.pivots].T for c in range(3)]
    _, _, D = xtc.d_kernels(w.grid_w, xi, calG, xtc.g_nu(phiP, w.n_occ))
    X = xtc.x_projector(w.grid_w, xi, calG, phiP, w.n_occ)
    E = energies.energies(W, D, X, phiP, dphiP, w.n_occ)
    return dict(phi=phi, dphi=dphi, res=res, xi=xi, xit=xit, lams=lams, W=W, calG=calG,
                phiP=phiP, dphiP=np.stack(dphiP), D=D, X=X, E=E)


@pytest.fixture(scope="module")
def h6():
    w = wl.h6_chain()
    return w, oracle_case(w)


def test_orbitals(P, h6):
    w, o = h6
    b = w.basis
    phi, dphi = P.isdf_eval_orbitals(cu(b.center), cu(b.powers, torch.int32), cu(b.exps),
                                     cu(b.coefs), cu(w.mo_coef), cu(w.grid_xyz))
    assert rel(host(phi), o["phi"]) < 1e-12
    assert rel(host(dphi), o["dphi"]) < 1e-12


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_pivots_bit_exact(P, h6, mode):
    w, o = h6
    ref = pivots.select(o["phi"], o["dphi"], w.grid_w, w.n_mu,
                        mode={0: "fused", 1: "scalar", 2: "gradient"}[mode])
    piv = P.isdf_points(cu(o["phi"]), cu(o["dphi"]), cu(w.grid_w), w.n_mu, mode)
    want = {0: ref.pivots, 1: ref.piv_s, 2: ref.piv_v}[mode]
    assert np.array_equal(host(piv), want)


@pytest.mark.parametrize("ranks", [(48, 60), (96, 0), (0, 40), (30, 100)])
def test_pivots_fixed_rank_bit_exact(P, h6, ranks):
    """The paper's fusion: each channel to its own rank, then the union."""
    w, o = h6
    ref = pivots.select_ranks(o["phi"], o["dphi"], w.grid_w, *ranks)
    piv = P.isdf_points_fixed_rank(cu(o["phi"]), cu(o["dphi"]), cu(w.grid_w), *ranks,
                                   allow_rank=True)
    assert np.array_equal(host(piv), ref.pivots)
    assert len(ref.pivots) <= sum(ranks)


def test_pivots_fixed_rank_three_points(P):
    """The hand-worked three-point cases of the fixed-rank fusion, on the GPU."""
    phi = np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 1.0]])
    dphi = np.zeros((3, 2, 3))
    dphi[0] = [[0.0, 2.0, 0.0], [0.0, 0.0, 1.0]]
    for ranks, want in (((1, 2), [2, 1]), ((2, 2), [2, 0, 1]), ((3, 2), [2, 0, 1]),
                        ((0, 2), [1, 2]), ((2, 0), [2, 0]), ((3, 3), [2, 0, 1])):
        piv = P.isdf_points_fixed_rank(cu(phi), cu(dphi), cu(np.ones(3)), *ranks, allow_rank=True)
        assert host(piv).tolist() == want, ranks


def test_pivots_rank_exhaustion(P):
    """3 s orbitals: the scalar channel has rank 6; asking for 50 stops at 6
    with ISDF_E_RANK, identically to the oracle."""
    w = wl.tiny_chain(n_atom=3, n_rad=16, n_ang=26, shells=(0,), seed=11)
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    ref = pivots.select(phi, dphi, w.grid_w, 50, mode="scalar")
    piv = P.isdf_points(cu(phi), cu(dphi), cu(w.grid_w), 50, 1, allow_rank=True)
    assert ref.rank_exhausted and np.array_equal(host(piv), ref.piv_s)


def test_fit(P, h6):
    """Backward error of the GPU's FP64 solves at 1e-10 (normal-equation
    residual against the oracle's Grams and right-hand sides), and forward
    agreement with the oracle within the Grams' condition number times the
    FP64 unit roundoff (kappa ~ 2e6 on this system)."""
    w, o = h6
    xi, xig, jit = P.isdf_fit(cu(o["phi"]), cu(o["dphi"]), cu(o["res"].pivots, torch.int32))
    assert np.allclose(jit, o["lams"])
    Gm = fit.grams(o["phi"], o["dphi"], o["res"].pivots)
    B = fit.rhs(o["phi"], o["dphi"], o["res"].pivots)
    X = np.concatenate([host(xi)[None], host(xig)])
    Xo = np.concatenate([o["xi"][None], o["xit"]])
    for c in range(4):
        G = Gm[c] + o["lams"][c] * np.eye(Gm.shape[1])
        back = np.linalg.norm(G @ X[c] - B[c]) / (np.linalg.norm(G) * np.linalg.norm(X[c]))
        kappa = np.linalg.cond(G)
        fwd = rel(X[c], Xo[c])
        print("fit channel", c, "backward error %.2e" % back, "cond %.2e" % kappa,
              "forward %.2e" % fwd)
        assert back < 1e-10, (c, back)
        assert fwd < max(1e-10, 8.0 * kappa * np.finfo(float).eps), (c, fwd, kappa)


def test_fit_jitter_policy(P, h6):
    """The jitter policy of isdf_options (Sec. IV.B's adaptive Tikhonov shift):
    396 pivots on 24 orbitals (300 distinct pair products) make the scalar Gram
    singular, so the unshifted factorisation fails; with no retries allowed the
    fit returns ISDF_E_NOT_PD, and with jitter_init 1e-8 the shift used is
    1e-8 10^k times the Gram's largest diagonal, for which the solve keeps a
    backward error of 1e-10."""
    from paper_2607_17314_b300 import _capi as C
    w, o = h6
    rng = np.random.default_rng(7)
    rest = np.setdiff1d(np.arange(w.n_g), o["res"].pivots)
    piv = np.concatenate([o["res"].pivots, rng.choice(rest, 300, replace=False)]).astype(np.int32)
    phi, dphi, pv = cu(o["phi"]), cu(o["dphi"]), cu(piv, torch.int32)
    with pytest.raises(C.IsdfError) as e:
        P.isdf_fit(phi, dphi, pv, max_jitter_tries=-1)
    assert e.value.status == C.ISDF_E_NOT_PD
    xi, _, jit = P.isdf_fit(phi, dphi, pv, jitter_init=1e-8)
    Gm = fit.grams(o["phi"], o["dphi"], piv)
    maxd = float(np.max(np.diag(Gm[0])))
    k = np.log10(jit[0] / (1e-8 * maxd))
    assert jit[0] > 0 and abs(k - round(k)) < 1e-9 and 0 <= round(k) <= 8, (jit[0], maxd)
    G = Gm[0] + jit[0] * np.eye(len(piv))
    X = host(xi)
    B = fit.rhs(o["phi"], o["dphi"], piv)[0]
    back = np.linalg.norm(G @ X - B) / (np.linalg.norm(G) * np.linalg.norm(X))
    assert back < 1e-10, back


def _jas(P, w):
    return P.jastrow_from(w.jastrow)


def test_w_fp64(P, h6):
    w, o = h6
    W, calG = P.tc_kernel_build(cu(w.grid_xyz), cu(w.grid_w), cu(o["xi"]), cu(o["xit"]),
                                _jas(P, w), "fp64")
    for c in range(4):
        assert rel(host(W[c]), o["W"][c]) < 1e-10, c
        assert rel(host(calG[c]), o["calG"][c]) < 1e-10, c


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6", "tf32x3"])
def test_w_tensor_core(P, h6, prec):
    w, o = h6
    W, calG = P.tc_kernel_build(cu(w.grid_xyz), cu(w.grid_w), cu(o["xi"]), cu(o["xit"]),
                                _jas(P, w), prec)
    errs = [rel(host(W[c]), o["W"][c]) for c in range(4)]
    gerrs = [rel(host(calG[c]), o["calG"][c]) for c in range(4)]
    print(prec, "W rel", errs, "calG rel", gerrs)
    # the error is dominated by the tensor core's FP32 accumulation, kept
    # short by folding every 384 inner points into an FP32 running sum;
    # both limb counts meet the 1e-5 bar
    assert max(errs) < 1e-5, errs


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_w_one_body_term(P, h6, prec):
    """The radial correlator plus the one-body cusp term of Eq. tau-def (H: Z = 1,
    N = 2 n_occ electrons): FP64 at 1e-10 and the tensor cores (multi-centre
    generator, the term in its inner-point-free part) at 1e-5 per channel,
    against the oracle's W on the same fitted factors."""
    w, o = h6
    jas = wl.with_chi(wl.radial_jastrow(w.xyz), [1.0], 2 * w.n_occ, beta=1.2)
    Wo, calGo = wbuild.build(w.grid_xyz, w.grid_w, o["xi"], o["xit"], jas)
    W, calG = P.tc_kernel_build(cu(w.grid_xyz), cu(w.grid_w), cu(o["xi"]), cu(o["xit"]),
                                P.jastrow_from(jas), prec)
    errs = [rel(host(W[c]), Wo[c]) for c in range(4)]
    gerrs = [rel(host(calG[c]), calGo[c]) for c in range(4)]
    print(prec, "one-body term: W rel", errs, "calG rel", gerrs)
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert max(errs) < tol and max(gerrs) < tol, (errs, gerrs)
    # the term changes W: it is not silently dropped
    assert min(rel(Wo[c], o["W"][c]) for c in range(4)) > 1e-3


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_w_streamed_from_host(P, h6, prec):
    """The streamed build (xi and xi~ in pinned host memory, bra batches of 1000
    outer points, ket batches of 1024 inner points: ragged tiles and a ragged
    last batch) against the oracle's W at 1e-5 per channel, and against the
    resident build at 5e-6."""
    w, o = h6
    J = _jas(P, w)
    xi_h = torch.as_tensor(o["xi"]).contiguous().pin_memory()
    xig_h = torch.as_tensor(o["xit"]).contiguous().pin_memory()
    g, wt = cu(w.grid_xyz), cu(w.grid_w)
    Ws = P.tc_kernel_build_streamed(g, wt, xi_h, xig_h, J, prec, bra=1000, ket=1024)
    Wr, _ = P.tc_kernel_build(g, wt, cu(o["xi"]), cu(o["xit"]), J, prec)
    errs = [rel(host(Ws[c]), o["W"][c]) for c in range(4)]
    diffs = [rel(host(Ws[c]), host(Wr[c])) for c in range(4)]
    print(prec, "streamed W rel vs oracle", errs, "vs resident", diffs)
    assert max(errs) < 1e-5, errs
    assert max(diffs) < 5e-6, diffs


def test_w_streamed_multi_centre(P):
    """The streamed build with the two-type multi-centre correlator and the
    one-body term on a small benzene grid (random xi, so W carries heavy
    cancellation): against the resident build at 5e-6 and the oracle at 1e-4."""
    atoms, xyz = wl.benzene()
    grid, wgt = wl.becke_grid(xyz, 6, 26)
    jas = wl.with_chi(wl.bh_jastrow(atoms, xyz, wl.BH_TERMS_C3, np.random.default_rng(11)),
                      [6.0, 1.0], 42)
    n_mu = 40
    xi = wl.seeded_matrix((n_mu, grid.shape[0]), 31, 1e-2)
    xit = wl.seeded_matrix((3, n_mu, grid.shape[0]), 32, 1e-2)
    Wo, _ = wbuild.build(grid, wgt, xi, xit, jas)
    Ws = P.tc_kernel_build_streamed(cu(grid), cu(wgt), torch.as_tensor(xi).pin_memory(),
                                    torch.as_tensor(xit).pin_memory(), P.jastrow_from(jas),
                                    "bf16x3", bra=300, ket=320)
    Wr, _ = P.tc_kernel_build(cu(grid), cu(wgt), cu(xi), cu(xit), P.jastrow_from(jas), "bf16x3")
    errs = [rel(host(Ws[c]), Wo[c]) for c in range(4)]
    diffs = [rel(host(Ws[c]), host(Wr[c])) for c in range(4)]
    print("streamed multi-centre W rel vs oracle", errs, "vs resident", diffs)
    assert max(diffs) < 5e-6, diffs
    assert max(errs) < 1e-4, errs


def test_w_tensor_core_single_cta(P, h6):
    """The single-CTA stage-1 kernel (128-row tiles), kept for the multi-centre
    correlator, on the radial correlator with two limbs (debug bit 1 selects it)."""
    from paper_2607_17314_b300 import api
    w, o = h6
    kb = api.KernelBuilder(cu(w.grid_xyz), cu(w.grid_w), cu(o["xi"]), cu(o["xit"]), _jas(P, w),
                           "bf16x3", debug_flags=2)
    kb()
    errs = [rel(host(kb.W[c]), o["W"][c]) for c in range(4)]
    assert max(errs) < 1e-5, errs


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_w_slices_additive(P, h6, prec):
    w, o = h6
    args = (cu(w.grid_xyz), cu(w.grid_w), cu(o["xi"]), cu(o["xit"]), _jas(P, w), prec)
    Wf, Gf = P.tc_kernel_build(*args)
    cut = 1717
    Wa, Ga = P.tc_kernel_build(*args, g_begin=0, g_end=cut)
    Wb, Gb = P.tc_kernel_build(*args, g_begin=cut, g_end=w.n_g)
    # tensor-core partials each carry their own accumulation rounding
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert rel(host(Wa + Wb), host(Wf)) < tol
    assert rel(host(torch.cat([Ga, Gb], dim=2)), host(Gf)) < tol


def test_xtc(P, h6):
    w, o = h6
    n_orb = w.n_orb
    D, Xp = P.xtc_density_contract(cu(o["phiP"]), w.n_occ, cu(o["xi"]), cu(w.grid_w),
                                   cu(o["calG"]), n_orb_x=n_orb)
    _, _, Dref = xtc.d_kernels(w.grid_w, o["xi"], o["calG"], xtc.g_nu(o["phiP"], w.n_occ))
    assert rel(host(D), Dref) < 1e-10
    Xfull = xtc.x_projector(w.grid_w, o["xi"], o["calG"], o["phiP"], w.n_occ)
    assert rel(host(Xp), xtc.pack_upper(Xfull)) < 1e-10


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_xtc_tensor_core(P, h6, prec):
    """D and X on the split-BF16 tensor-core GEMMs."""
    w, o = h6
    n_orb = w.n_orb
    D, Xp = P.xtc_density_contract(cu(o["phiP"]), w.n_occ, cu(o["xi"]), cu(w.grid_w),
                                   cu(o["calG"]), n_orb_x=n_orb, precision=prec)
    _, _, Dref = xtc.d_kernels(w.grid_w, o["xi"], o["calG"], xtc.g_nu(o["phiP"], w.n_occ))
    assert rel(host(D), Dref) < 1e-5
    Xfull = xtc.x_projector(w.grid_w, o["xi"], o["calG"], o["phiP"], w.n_occ)
    xerr = rel(host(Xp), xtc.pack_upper(Xfull))
    print(prec, "X rel", xerr)
    assert xerr < 1e-5


def test_xtc_tensor_core_chunks(P):
    """Several 32768-point grid chunks with a ragged tail (n_g = 70001) and
    n_mu = 200 (two M tiles, ragged): seeded standard-normal factors."""
    n_mu, n_g, n_orb, n_occ = 200, 70001, 12, 5
    phiP = wl.seeded_matrix((n_mu, n_orb), 11)
    xi = wl.seeded_matrix((n_mu, n_g), 12)
    calG = wl.seeded_matrix((3, n_mu, n_g), 13)
    wg = np.abs(wl.seeded_matrix((n_g,), 14)) + 0.1
    D, _ = P.xtc_density_contract(cu(phiP), n_occ, cu(xi), cu(wg), cu(calG), precision="bf16x6")
    _, _, Dref = xtc.d_kernels(wg, xi, calG, xtc.g_nu(phiP, n_occ))
    assert rel(host(D), Dref) < 1e-5


def test_energies_fp64(P, h6):
    w, o = h6
    Xp = xtc.pack_upper(o["X"])
    E = P.tc_energies(cu(o["W"]), cu(o["D"]), cu(Xp), cu(o["phiP"]), cu(o["dphiP"]), w.n_occ)
    ref = o["E"]
    for got, key in zip(E, ("E_K", "E_dU", "E0")):
        assert abs(got - ref[key]) <= 1e-10 * abs(ref[key]) + 1e-14, (key, got, ref[key])


def pivots_against_oracle(phi_gpu, dphi_gpu, w, n_mu, piv_gpu, o):
    """Bit-exact pivots on identical inputs, and a proven near tie for any
    index that differs from the oracle's selection on its own orbitals.
    Returns a one-line account of what was checked."""
    same_in = pivots.select(phi_gpu, dphi_gpu, w, n_mu)
    assert np.array_equal(piv_gpu, same_in.pivots), "GPU pivots differ on identical inputs"
    ref = o["res"]
    if np.array_equal(piv_gpu, ref.pivots):
        return "pivots bit-exact (identical inputs and oracle orbitals)"
    # the GPU's orbitals differ from the oracle's in the last bits: the first
    # divergent step of each channel must be a tie within that rounding
    notes = []
    for ch, a, b in (("scalar", ref.piv_s, same_in.piv_s), ("gradient", ref.piv_v, same_in.piv_v)):
        j, gap = pivots.tie_margin(o["phi"], o["dphi"], w, a, b, ch)
        if j is not None:
            assert gap <= 1e-10, (ch, j, gap)
            notes.append(f"{ch} step {j} near tie (gap {gap:.1e})")
    return "pivots bit-exact on identical inputs; " + "; ".join(notes)


def oracle_energies(w, phi, dphi, piv, xi, xit):
    """The oracle's W, D, X and energies from given orbitals, pivots and fit."""
    W, calG = wbuild.build(w.grid_xyz, w.grid_w, xi, xit, w.jastrow)
    phiP = xtc.pivot_factors(phi, piv)
    _, _, D = xtc.d_kernels(w.grid_w, xi, calG, xtc.g_nu(phiP, w.n_occ))
    X = xtc.x_projector(w.grid_w, xi, calG, phiP, w.n_occ)
    return energies.energies(W, D, X, phiP, [dphi[c][:, piv].T for c in range(3)], w.n_occ)


@pytest.mark.parametrize("prec", ["fp64", "bf16x6", "bf16x3"])
def test_end_to_end(P, h6, prec):
    """Full path on the GPU (a1 -> a6).  Pivots bit-exact on identical inputs
    (near ties proven where the oracle's own orbitals flip one); energies
    against the oracle evaluated on the GPU's orbitals, pivots and fit at
    1e-10 relative (FP64) or 1e-6 Ha (tensor cores), and against the
    oracle's whole chain at 1e-6 Ha."""
    from paper_2607_17314_b300 import pipeline
    w, o = h6
    b = w.basis
    inp = pipeline.upload(b.center, b.powers, b.exps, b.coefs, w.mo_coef, w.grid_xyz, w.grid_w,
                          w.n_mu, w.n_occ, _jas(P, w))
    out = pipeline.run(inp, precision=prec)
    piv = host(out["pivots"])
    phi_g, dphi_g = host(out["phi"]), host(out["dphi"])
    print(pivots_against_oracle(phi_g, dphi_g, w.grid_w, w.n_mu, piv, o))
    E_same = oracle_energies(w, phi_g, dphi_g, piv, host(out["xi"]), host(out["xig"]))
    for got, key in zip(out["E"], ("E_K", "E_dU", "E0")):
        tol = 1e-10 * abs(E_same[key]) + 1e-14 if prec == "fp64" else 1e-6
        assert abs(got - E_same[key]) <= tol, (key, got, E_same[key])
        assert abs(got - o["E"][key]) <= 1e-6, (key, got, o["E"][key])


def test_ragged_small_system(P):
    """n_g = 2 x 9 x 14 = 252 (ragged against 128 and 32), n_mu = 13."""
    w = wl.tiny_chain(n_atom=2, n_rad=9, n_ang=14, shells=(0, 1), n_mu=13, seed=21)
    o = oracle_case(w)
    args = (cu(w.grid_xyz), cu(w.grid_w), cu(o["xi"]), cu(o["xit"]), _jas(P, w))
    W64, G64 = P.tc_kernel_build(*args, "fp64")
    assert max(rel(host(W64[c]), o["W"][c]) for c in range(4)) < 1e-10
    W16, _ = P.tc_kernel_build(*args, "bf16x6")
    assert max(rel(host(W16[c]), o["W"][c]) for c in range(4)) < 1e-5


_BENZ = {}


def _benzene_case(jscale):
    if jscale not in _BENZ:
        w = wl.benzene_small(jscale=jscale)
        _BENZ[jscale] = (w, oracle_case(w))
    return _BENZ[jscale]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("jscale", [0.05, 0.5])
def test_w_tensor_core_bh(P, prec, jscale):
    """Multi-centre (e-e, e-n, e-e-n) correlator of the benzene workload on the
    tensor-core path: 12 centres, two types, 1008 points (ragged in both grid
    directions), N_mu = 64.  jscale = 0.5 makes the free terms dominate."""
    w, o = _benzene_case(jscale)
    W, calG = P.tc_kernel_build(cu(w.grid_xyz), cu(w.grid_w), cu(o["xi"]), cu(o["xit"]),
                                _jas(P, w), prec)
    errs = [rel(host(W[c]), o["W"][c]) for c in range(4)]
    gerr = [rel(host(calG[c]), o["calG"][c]) for c in range(4)]
    print(prec, jscale, "W", errs, "calG", gerr)
    assert max(errs) < 1e-5, errs
    assert max(gerr) < 1e-5, gerr


@pytest.mark.parametrize("terms", ["c4", "deg3"])
def test_w_tensor_core_bh_forms(P, terms):
    """The other generator forms: two E-exponent groups with degree 3 (the
    28-term set), and one group with degree 3."""
    jt = wl.bh_terms_c4() if terms == "c4" else [(3, 1, 2), (1, 0, 0), (0, 0, 3), (2, 1, 0)]
    w = wl.tiny_chain(n_atom=3, n_rad=8, n_ang=14, shells=(0, 1), n_mu=20, seed=5,
                      jkind="bh", jterms=jt)
    w.jastrow.coef[:] *= 10.0
    o = oracle_case(w)
    args = (cu(w.grid_xyz), cu(w.grid_w), cu(o["xi"]), cu(o["xit"]), _jas(P, w))
    W, calG = P.tc_kernel_build(*args, "bf16x6")
    errs = [rel(host(W[c]), o["W"][c]) for c in range(4)]
    print(terms, errs)
    assert max(errs) < 1e-5, errs


def test_w_tensor_core_bh_slices(P):
    """Outer-grid slices of the multi-centre build are additive."""
    w, o = _benzene_case(0.05)
    args = (cu(w.grid_xyz), cu(w.grid_w), cu(o["xi"]), cu(o["xit"]), _jas(P, w))
    n_g = w.grid_xyz.shape[0]
    Wsum = 0
    for a, b in ((0, 300), (300, 700), (700, n_g)):
        Ws, _ = P.tc_kernel_build(*args, "bf16x3", g_begin=a, g_end=b)
        Wsum = Wsum + host(Ws)
    assert max(rel(Wsum[c], o["W"][c]) for c in range(4)) < 1e-5


def test_bh_jastrow_fp64(P):
    """Multi-centre Boys-Handy correlator (e-e, e-n, e-e-n terms) on the FP64 path."""
    w = wl.tiny_chain(n_atom=3, n_rad=8, n_ang=14, shells=(0, 1), n_mu=20, seed=5,
                      jkind="bh", jterms=wl.bh_terms_c4())
    o = oracle_case(w)
    W, calG = P.tc_kernel_build(cu(w.grid_xyz), cu(w.grid_w), cu(o["xi"]), cu(o["xit"]),
                                _jas(P, w), "fp64")
    for c in range(4):
        assert rel(host(W[c]), o["W"][c]) < 1e-10, c


def test_zero_jastrow_fp64(P, h6):
    w, o = h6
    J = _jas(P, w)
    J.cusp = 0
    W, calG = P.tc_kernel_build(cu(w.grid_xyz), cu(w.grid_w), cu(o["xi"]), cu(o["xit"]), J, "fp64")
    assert float(W.abs().max()) == 0.0 and float(calG.abs().max()) == 0.0


@pytest.fixture(scope="module")
def h6_four_index(h6):
    """The oracle's K and DeltaU over every orbital index of the H6 case."""
    w, o = h6
    idx = np.arange(w.n_orb)
    K = energies.k_tensor(o["W"], o["phiP"], list(o["dphiP"]), idx)
    dU = energies.du_tensor(o["D"], o["X"], o["phiP"], idx)
    return K, dU


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_two_body_panels(P, h6, h6_four_index, prec):
    """K and DeltaU over all n_orb^2 x n_orb^2 composite entries, built panel by
    panel (three panels, the last ragged), against the oracle's four-index
    tensors (Eqs. K-recombine-final, deltaU-four)."""
    from paper_2607_17314_b300 import api
    w, o = h6
    K, dU = h6_four_index
    n = w.n_orb
    Kref = K.transpose(0, 2, 1, 3).reshape(n * n, n * n)      # [(p,r)][(q,s)]
    Uref = dU.transpose(0, 2, 1, 3).reshape(n * n, n * n)
    args = (cu(o["W"]), cu(o["D"]), cu(xtc.pack_upper(o["X"])), cu(o["phiP"]), cu(o["dphiP"]))
    cuts = [0, 250, 500, n * n]
    Kg, Ug = [], []
    for a, b in zip(cuts, cuts[1:]):
        kp, up = api.tc_two_body_panel(*args, a, b, precision=prec)
        Kg.append(host(kp))
        Ug.append(host(up))
    Kg, Ug = np.concatenate(Kg), np.concatenate(Ug)
    ek = float(np.max(np.abs(Kg - Kref)) / np.max(np.abs(Kref)))
    eu = float(np.max(np.abs(Ug - Uref)) / np.max(np.abs(Uref)))
    print(prec, "K max err / max %.2e" % ek, "DeltaU %.2e" % eu,
          "rel Frobenius", rel(Kg, Kref), rel(Ug, Uref))
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert ek < tol and eu < tol


def test_xtc_one_body(P, h6, h6_four_index):
    """Delta h, f^xTC and E0 over every orbital pair (Eqs. xtc-deltah, xtc-fock,
    xtc-const) against the oracle's contractions of the four-index tensors."""
    from paper_2607_17314_b300 import api
    w, o = h6
    K, dU = h6_four_index
    occ = np.arange(w.n_occ)
    dh_ref = energies.delta_h(dU, occ)
    f_ref = energies.fock_xtc(K, dU, occ)
    e0_ref = energies.e0_xtc(dh_ref, occ)
    dh, f, e0 = api.tc_xtc_one_body(cu(o["W"]), cu(o["D"]), cu(xtc.pack_upper(o["X"])),
                                    cu(o["phiP"]), cu(o["dphiP"]), w.n_occ)
    assert rel(host(dh), dh_ref) < 1e-10
    assert rel(host(f), f_ref) < 1e-10
    assert abs(e0 - e0_ref) <= 1e-10 * abs(e0_ref)
    # and E0 agrees with the occupied-block energies call
    assert abs(e0 - o["E"]["E0"]) <= 1e-10 * abs(e0_ref)
