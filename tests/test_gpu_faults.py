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
