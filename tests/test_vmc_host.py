"""Host logic of the VMC front end (Sec. II.C's reference-variance protocol):
the adaptive Tikhonov shift of VmcOptimizer and the Polyak-Ruppert window of
vmc_schedule, with the device calls replaced by fakes on CPU tensors.  In the
fakes the local energies are theta itself and the clipped variance is
|theta|^2, so a scripted Gauss-Newton proposal decides every accept or reject."""
import numpy as np
import pytest
import torch

from paper_2607_17314_b300 import api


class FakeDevice:
    """Stand-ins for the five VMC calls; `proposals` are the Gauss-Newton steps
    the fake returns in turn, `thetas_seen` records theta at every sample call."""

    def __init__(self, proposals):
        self.proposals = [torch.as_tensor(p, dtype=torch.float64) for p in proposals]
        self.calls = {"eloc": 0, "gn": 0, "sample": 0}
        self.thetas_seen = []
        self.theta = None

    def local_energy(self, basis, mo_coef, n_occ, walkers, jastrow, charges, theta, h, grad=True):
        self.calls["eloc"] += 1
        E = theta.clone()
        return E if not grad else (E, torch.zeros((theta.numel(), theta.numel()), dtype=torch.float64))

    def objective(self, E):
        return torch.tensor([0.0, float(E @ E), 0.0, 0.0], dtype=torch.float64)

    def gn_step(self, E, dE, lam, eta, theta=None):
        step = self.proposals[self.calls["gn"]]
        self.calls["gn"] += 1
        theta += step
        return step, torch.tensor([0.0, float(E @ E), 0.0, 0.0], dtype=torch.float64)

    def sample(self, basis, mo_coef, n_occ, walkers, normals, uniforms, sigma):
        self.calls["sample"] += 1
        self.thetas_seen.append(self.theta.clone())
        return 7

    @staticmethod
    def polyak(theta, avg, k):
        if k == 1:
            avg.copy_(theta)
        else:
            avg += (theta - avg) / k
        return avg


@pytest.fixture
def fake(monkeypatch):
    def install(proposals):
        f = FakeDevice(proposals)
        monkeypatch.setattr(api, "isdf_vmc_local_energy", f.local_energy)
        monkeypatch.setattr(api, "isdf_vmc_objective", f.objective)
        monkeypatch.setattr(api, "isdf_vmc_gn_step", f.gn_step)
        monkeypatch.setattr(api, "isdf_vmc_sample", f.sample)
        monkeypatch.setattr(api, "isdf_vmc_polyak", f.polyak)
        return f
    return install


def test_optimizer_keeps_only_downhill_steps(fake):
    """A step that lowers the variance is kept and lam /= 3; one that raises it
    leaves theta and the recorded variance alone and lam *= 10."""
    f = fake([[-0.5, 0.0], [1.0, 1.0], [0.0, -1.0]])
    theta = torch.tensor([1.0, 1.0], dtype=torch.float64)
    opt = api.VmcOptimizer(None, None, 1, None, None, None, theta, lam=1e-2, eta=0.5)
    assert opt.var == 2.0
    var, lam, ok = opt.step()
    assert ok and var == 0.25 + 1.0 and lam == pytest.approx(1e-2 / 3)
    assert torch.equal(theta, torch.tensor([0.5, 1.0], dtype=torch.float64))
    var, lam, ok = opt.step()
    assert not ok and var == 1.25 and lam == pytest.approx(1e-1 / 3)
    assert torch.equal(theta, torch.tensor([0.5, 1.0], dtype=torch.float64))
    var, lam, ok = opt.step()
    assert ok and var == 0.25 and lam == pytest.approx(1e-1 / 9)
    assert torch.equal(theta, torch.tensor([0.5, 0.0], dtype=torch.float64))
    assert f.calls["gn"] == 3


def test_optimizer_clamps_the_shift(fake):
    """lam stays within [lam_min, lam_max]: three uphill steps from lam = 0.5
    give 5, 20 (50 clamped), 20; six downhill steps then give 20/3, 20/9,
    20/27, 20/81 and 0.1 twice (clamped)."""
    fake([[1.0]] * 3 + [[-0.1]] * 6)
    theta = torch.tensor([1.0], dtype=torch.float64)
    opt = api.VmcOptimizer(None, None, 1, None, None, None, theta, lam=0.5, lam_min=0.1,
                           lam_max=20.0)
    out = [opt.step() for _ in range(9)]
    assert [o[2] for o in out] == [False] * 3 + [True] * 6
    assert np.allclose([o[1] for o in out],
                       [5.0, 20.0, 20.0, 20 / 3, 20 / 9, 20 / 27, 20 / 81, 0.1, 0.1], rtol=1e-15)
    assert float(theta) == pytest.approx(0.4, abs=1e-15)


@pytest.mark.parametrize("n_warm,n_refine,window", [(2, 5, 3), (0, 4, 4), (3, 3, 1)])
def test_schedule_averages_the_last_window_steps(fake, n_warm, n_refine, window):
    """Every step samples, then steps; the returned average is the mean of theta
    after each of the last `window` steps, and the history carries one entry per
    step with the acceptance ratio accepted / (sweeps N n_w)."""
    n = n_warm + n_refine
    rng = np.random.default_rng(n_warm * 10 + window)
    props = -np.abs(rng.uniform(0.01, 0.05, (n, 3)))  # always downhill from theta > 0.5
    f = fake(props)
    theta = torch.tensor([2.0, 1.5, 1.0], dtype=torch.float64)
    f.theta = theta
    walkers = torch.zeros((4, 2, 3), dtype=torch.float64)
    gen = torch.Generator()
    gen.manual_seed(0)
    avg, hist = api.vmc_schedule(None, None, 1, walkers, None, None, theta, n_warm=n_warm,
                                 n_refine=n_refine, window=window, sweeps=3, sigma=0.5,
                                 generator=gen)
    assert len(hist) == n and all(h[2] for h in hist)
    assert all(h[3] == pytest.approx(7 / (3 * 2 * 4)) for h in hist)
    traj = np.array([2.0, 1.5, 1.0]) + np.cumsum(props, axis=0)   # theta after each step
    assert np.allclose(theta.numpy(), traj[-1])
    assert np.allclose(avg.numpy(), traj[-window:].mean(axis=0), rtol=1e-14, atol=0)
    assert f.calls["sample"] == n
    # each sample call sees theta as the previous step left it
    assert np.allclose(f.thetas_seen[1].numpy(), traj[0])


def test_polyak_rejects_mismatched_sizes():
    with pytest.raises(ValueError, match="avg has 2 values"):
        api.isdf_vmc_polyak(torch.zeros(3, dtype=torch.float64), torch.zeros(2, dtype=torch.float64), 1)
