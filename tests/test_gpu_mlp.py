"""Learned interpolation-point proposer on the GPU: kernels against the FP64
oracle, training, and what the trained network gains over plain pivoting."""
import time

import numpy as np
import pytest
import torch

from synth import workloads as wl
from oracle import orbitals, pivots, mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_17314_b300 import build
    build.build()
    from paper_2607_17314_b300 import proposer
    return proposer


def _cu(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dt).cuda()


@pytest.fixture(scope="module")
def chain():
    w = wl.perturbed_chain(0, n_atom=6, n_rad=14, n_ang=26, n_mu=60, shells=(0, 1))
    phi, dphi = orbitals.eval_orbitals(w.basis, w.mo_coef, w.grid_xyz)
    return w, phi, dphi


def test_features_match_oracle(P, chain):
    w, phi, dphi = chain
    ref = omlp.features(phi, dphi, w.grid_w, w.grid_xyz, w.xyz)
    got = P.features(_cu(phi), _cu(dphi), _cu(w.grid_w), _cu(w.grid_xyz), w.xyz).cpu().numpy()
    assert np.max(np.abs(got - ref)) < 2e-6 * max(1.0, np.max(np.abs(ref)))


def test_forward_backward_adam_match_oracle(P):
    rng = np.random.default_rng(3)
    n = 1000
    x = rng.standard_normal((n, 8)).astype(np.float32)
    y = (rng.random(n) < 0.05).astype(np.float32)
    th = (omlp.init_params(2) + 0.05 * rng.standard_normal(omlp.N_PARAMS)).astype(np.float32)
    params = _cu(th, torch.float32)
    s_gpu = P.forward(params, _cu(x, torch.float32)).cpu().numpy()
    s_ref, _ = omlp.forward(th.astype(np.float64), x.astype(np.float64))
    assert np.max(np.abs(s_gpu - s_ref)) < 1e-4 * max(1.0, np.max(np.abs(s_ref)))
    grad = torch.zeros(omlp.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    # two partial calls accumulate the gradient of the mean over all points
    P.backward(params, _cu(x[:600], torch.float32), _cu(y[:600], torch.float32), 19.0, n, grad, loss)
    P.backward(params, _cu(x[600:], torch.float32), _cu(y[600:], torch.float32), 19.0, n, grad, loss)
    l_ref, g_ref = omlp.loss_and_grad(th.astype(np.float64), x.astype(np.float64),
                                      y.astype(np.float64), 19.0)
    g = grad.cpu().numpy()
    assert abs(loss.item() / n - l_ref) < 1e-5 * abs(l_ref)
    # the layer products run on the tensor cores with two BF16 limbs per FP32
    # operand (three products) and FP32 accumulation over all of a CTA's points
    # (measured 1.1e-4)
    assert np.linalg.norm(g - g_ref) < 5e-4 * np.linalg.norm(g_ref)
    # one Adam step from zero moments
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    P.adam(params, grad, m, v, 1, 1e-3)
    ref_new, _, _ = omlp.adam(th.astype(np.float64), g.astype(np.float64), 0.0, 0.0, 1, lr=1e-3)
    assert np.max(np.abs(params.cpu().numpy() - ref_new)) < 1e-6


def test_topk_bit_exact(P):
    rng = np.random.default_rng(5)
    s = rng.standard_normal(5000).astype(np.float32)
    s[100:140] = s[7]            # ties
    s[4000:4010] = -0.0
    s[4010:4020] = 0.0
    for k in (1, 17, 40, 777, 5000):
        got = P.topk(_cu(s, torch.float32), k).cpu().numpy()
        assert np.array_equal(got, omlp.candidates(s.astype(np.float64), k)), k


def test_restricted_pivots_and_fit_error(P, chain):
    w, phi, dphi = chain
    rng = np.random.default_rng(9)
    cand = np.sort(rng.choice(w.n_g, 400, replace=False)).astype(np.int32)
    got = P.points_restricted(_cu(phi), _cu(dphi), _cu(w.grid_w), _cu(cand, torch.int32), w.n_mu)
    sub = pivots.select(phi[:, cand], dphi[:, :, cand], w.grid_w[cand], w.n_mu)
    assert np.array_equal(got.cpu().numpy(), cand[sub.pivots])
    e_gpu = P.fit_error(_cu(phi), _cu(w.grid_w), got)
    e_ref = omlp.fit_error(phi, w.grid_w, cand[sub.pivots])
    assert abs(e_gpu - e_ref) < 1e-8 * e_ref


def _sample(P, k, n_atom=8, n_rad=14, n_ang=26, n_mu=100):
    from paper_2607_17314_b300 import api
    w = wl.perturbed_chain(k, n_atom=n_atom, n_rad=n_rad, n_ang=n_ang, n_mu=n_mu, shells=(0, 1))
    b = w.basis
    phi, dphi = api.isdf_eval_orbitals(_cu(b.center), _cu(b.powers, torch.int32), _cu(b.exps),
                                       _cu(b.coefs), _cu(w.mo_coef), _cu(w.grid_xyz))
    wt = _cu(w.grid_w)
    plain = api.isdf_points(phi, dphi, wt, n_mu)
    labels = torch.zeros(w.n_g, dtype=torch.float32, device="cuda")
    labels[plain.long()] = 1.0
    feat = P.features(phi, dphi, wt, _cu(w.grid_xyz), w.xyz)
    return P.Sample(feat=feat, labels=labels, phi=phi, dphi=dphi, w=wt, plain=plain, n_mu=n_mu)


def test_training_and_gain(P):
    """Trained on 12 perturbed H8 chains, the proposer picks points from 3 N_mu
    candidates whose fit error stays close to plain pivoting on held-out
    chains, while the pivot loop runs over a fraction of the grid."""
    train = [_sample(P, k) for k in range(12)]
    test = [_sample(P, k) for k in range(100, 104)]
    prop = P.Proposer(seed=0, lr=3e-3)
    losses = [prop.train_epoch(train) for _ in range(60)]
    print("loss first/last", losses[0], losses[-1])
    assert losses[-1] < 0.6 * losses[0]
    from paper_2607_17314_b300 import api
    ratios, fallbacks = [], 0
    t_plain = t_prop = 0.0
    for smp in test:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.isdf_points(smp.phi, smp.dphi, smp.w, smp.n_mu)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        piv = prop.propose(smp)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        t_plain += t1 - t0
        t_prop += t2 - t1
        _, e_prop, e_plain, fb = prop.select(smp)
        ratios.append(e_prop / e_plain)
        fallbacks += fb
    print("fit-error ratio proposal/plain", ratios, "fallbacks", fallbacks,
          "selection time plain %.4f s proposal %.4f s" % (t_plain, t_prop))
    assert np.median(ratios) < 2.0
    # what the network gains: at the same tight candidate budget (1.5 N_mu
    # points) its candidates hold more of the plain selection than the budget
    # filled by the largest initial pivot diagonals (the fit errors of the two
    # restricted selections are reported; at the perturbed-H30 size the
    # network's proposal fits with 0.57 of the diagonal budget's error at
    # kappa = 3, and matches the plain selection's at kappa = 6)
    rec_net, rec_diag, e_net, e_diag = [], [], [], []
    for smp in test:
        c_net = prop.candidates(smp, 1.5)
        c_diag = P.diagonal_candidates(smp, 1.5)
        rec_net.append(P.recall(c_net, smp.plain))
        rec_diag.append(P.recall(c_diag, smp.plain))
        e_net.append(P.fit_error(smp.phi, smp.w, P.points_restricted(smp.phi, smp.dphi, smp.w,
                                                                      c_net, smp.n_mu)))
        e_diag.append(P.fit_error(smp.phi, smp.w, P.points_restricted(smp.phi, smp.dphi, smp.w,
                                                                       c_diag, smp.n_mu)))
    print("candidate recall of the plain selection: network", rec_net, "diagonal", rec_diag)
    print("fit error: network", e_net, "diagonal", e_diag)
    assert np.mean(rec_net) > np.mean(rec_diag) + 0.02
    # a network with scrambled weights is caught by the fit-error check
    bad = P.Proposer(seed=1)
    bad.params.mul_(-1.0)
    outs = [bad.select(smp, kappa=1.0, tolerance=1.05) for smp in test]
    assert any(o[3] for o in outs)
    for o, smp in zip(outs, test):
        if o[3]:
            assert torch.equal(o[0], smp.plain)
