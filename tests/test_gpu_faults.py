"""Fault paths on the GPU without a GPU fault: a bounded wait that nothing
satisfies returns ISDF_E_TIMEOUT, and the context stays usable."""
import numpy as np
import pytest
import torch

from synth import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_17314_b300 import build
    build.build()
    from paper_2607_17314_b300 import api
    return api


def _inputs(n_mu=40, seed=3):
    w = wl.tiny_chain(n_atom=2, n_rad=10, n_ang=14, shells=(0, 1), seed=seed)
    gen = np.random.default_rng(seed)
    xi = gen.standard_normal((n_mu, w.n_g)) * 1e-2
    xig = gen.standard_normal((3, n_mu, w.n_g)) * 1e-2
    c = lambda a: torch.as_tensor(a).cuda()
    return w, c(w.grid_xyz), c(w.grid_w), c(xi), c(xig)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_producer_stall_times_out_and_context_survives(api, prec):
    from paper_2607_17314_b300 import _capi as C
    w, g, wt, xi, xig = _inputs()
    J = api.jastrow_from(w.jastrow)
    bad = api.KernelBuilder(g, wt, xi, xig, J, prec, debug_flags=1)
    st = bad(allow_timeout=True)
    assert st == C.ISDF_E_TIMEOUT
    assert b"wait expired" in C.load().isdf_last_error()
    # the same context keeps working: a normal build matches the FP64 path
    W, _ = api.tc_kernel_build(g, wt, xi, xig, J, prec)
    W64, _ = api.tc_kernel_build(g, wt, xi, xig, J, "fp64")
    err = float(torch.linalg.norm(W - W64) / torch.linalg.norm(W64))
    assert err < 1e-4, err


def test_wait_limit_option(api):
    """isdf_options.wait_limit_ms bounds the device waits: the stalled build
    returns ISDF_E_TIMEOUT well before the default 2 s limit would expire."""
    import time
    from paper_2607_17314_b300 import _capi as C
    w, g, wt, xi, xig = _inputs()
    J = api.jastrow_from(w.jastrow)
    bad = api.KernelBuilder(g, wt, xi, xig, J, "bf16x3", debug_flags=1, wait_limit_ms=50)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = bad(allow_timeout=True)
    dt = time.perf_counter() - t0
    assert st == C.ISDF_E_TIMEOUT
    assert dt < 1.0, dt
    W, _ = api.tc_kernel_build(g, wt, xi, xig, J, "bf16x3")
    assert bool(torch.isfinite(W).all())
    with pytest.raises(C.IsdfError) as e:
        api.KernelBuilder(g, wt, xi, xig, J, "bf16x3", wait_limit_ms=-1)()
    assert e.value.status == C.ISDF_E_ARG


def test_bad_arguments_rejected_before_launch(api):
    from paper_2607_17314_b300 import _capi as C
    w, g, wt, xi, xig = _inputs()
    J = api.jastrow_from(w.jastrow)
    with pytest.raises(C.IsdfError) as e:
        api.tc_kernel_build(g, wt, xi, xig, J, "bf16x6", g_begin=5, g_end=3)
    assert e.value.status == C.ISDF_E_ARG
    # a term outside the tensor-core generator's polynomial form (m = 4)
    Jbh = api.jastrow_from(wl.bh_jastrow(w.atoms, w.xyz, [(4, 0, 0)], np.random.default_rng(0)))
    with pytest.raises(C.IsdfError) as e:
        api.tc_kernel_build(g, wt, xi, xig, Jbh, "bf16x6")
    assert e.value.status == C.ISDF_E_ARG


# ---------------------------------------------------------------- host-injected bad inputs
# Each case plants a NaN, an Inf or an out-of-range index in an input on the
# host.  The kernels never dereference an out-of-range index (the gather
# writes a quiet NaN instead), so nothing faults; the calls that synchronise
# report the problem by status.

def _orbital_case():
    from oracle import orbitals
    w = wl.tiny_chain(n_atom=2, n_rad=10, n_ang=14, shells=(0, 1), n_mu=16, seed=7)
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    c = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    return w, c(phi), c(dphi), c(w.grid_w)


def _status(fn):
    from paper_2607_17314_b300 import _capi as C
    try:
        fn()
    except C.IsdfError as e:
        return e.status
    return C.ISDF_OK


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_pivot_inputs(api, bad):
    from paper_2607_17314_b300 import _capi as C
    w, phi, dphi, wt = _orbital_case()
    wt2 = wt.clone()
    wt2[17] = bad
    assert _status(lambda: api.isdf_points(phi, dphi, wt2, w.n_mu)) == C.ISDF_E_NONFINITE
    assert _status(lambda: api.isdf_points_fixed_rank(phi, dphi, wt2, 4, 4)) == C.ISDF_E_NONFINITE
    dphi2 = dphi.clone()
    dphi2[2, 1, 5] = bad
    assert _status(lambda: api.isdf_points(phi, dphi2, wt, w.n_mu)) == C.ISDF_E_NONFINITE
    # the same context keeps working
    assert api.isdf_points(phi, dphi, wt, w.n_mu).numel() == w.n_mu


def test_nonfinite_fit_and_kernel_build(api):
    from paper_2607_17314_b300 import _capi as C
    w, phi, dphi, wt = _orbital_case()
    piv = api.isdf_points(phi, dphi, wt, w.n_mu)
    phi2 = phi.clone()
    phi2[0, 3] = float("nan")
    assert _status(lambda: api.isdf_fit(phi2, dphi, piv)) == C.ISDF_E_NONFINITE
    xi, xig, _ = api.isdf_fit(phi, dphi, piv)
    J = api.jastrow_from(w.jastrow)
    g = torch.as_tensor(w.grid_xyz).cuda()
    xi2 = xi.clone()
    xi2[1, 9] = float("inf")
    for prec in ("fp64", "bf16x3", "bf16x6"):
        assert _status(lambda: api.tc_kernel_build(g, wt, xi2, xig, J, prec)) == \
            C.ISDF_E_NONFINITE, prec
    W, calG = api.tc_kernel_build(g, wt, xi, xig, J, "bf16x3")
    phiP, dphiP = api.isdf_gather_pivots(phi, dphi, piv)
    calG2 = calG.clone()
    calG2[0, 2, 11] = float("nan")
    for prec in ("bf16x3", "bf16x6"):
        assert _status(lambda: api.xtc_density_contract(phiP, w.n_occ, xi, wt, calG2, w.n_occ,
                                                        precision=prec)) == C.ISDF_E_NONFINITE
    D, Xp = api.xtc_density_contract(phiP, w.n_occ, xi, wt, calG, w.n_occ)
    W2 = W.clone()
    W2[3, 0, 0] = float("nan")
    assert _status(lambda: api.tc_energies(W2, D, Xp, phiP, dphiP, w.n_occ)) == C.ISDF_E_NONFINITE
    assert all(np.isfinite(api.tc_energies(W, D, Xp, phiP, dphiP, w.n_occ)))


@pytest.mark.parametrize("bad_index", [-1, "n_g", 1 << 30])
def test_out_of_range_indices(api, bad_index):
    from paper_2607_17314_b300 import _capi as C, proposer
    w, phi, dphi, wt = _orbital_case()
    n_g = phi.shape[1]
    bad = n_g if bad_index == "n_g" else bad_index
    piv = api.isdf_points(phi, dphi, wt, w.n_mu)
    piv2 = piv.clone()
    piv2[5] = bad
    assert _status(lambda: api.isdf_fit(phi, dphi, piv2)) == C.ISDF_E_ARG
    assert _status(lambda: proposer.fit_error(phi, wt, piv2)) == C.ISDF_E_ARG
    # the asynchronous gather cannot report: the bad row becomes NaN
    phiP, dphiP = api.isdf_gather_pivots(phi, dphi, piv2)
    assert bool(torch.isnan(phiP[5]).all()) and bool(torch.isnan(dphiP[:, 5]).all())
    good = torch.cat([torch.arange(0, 5), torch.arange(6, phiP.shape[0])]).cuda()
    ref, _ = api.isdf_gather_pivots(phi, dphi, piv)
    assert torch.equal(phiP[good], ref[good])
    cand = torch.arange(0, n_g, 3, dtype=torch.int32, device="cuda")
    cand[2] = bad
    assert _status(lambda: proposer.points_restricted(phi, dphi, wt, cand, 8)) == C.ISDF_E_ARG
