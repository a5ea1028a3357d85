"""The seeded synthetic workloads build with the sizes of the configurations
they stand in for, positive quadrature weights and orthonormal orbitals."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from synth import workloads as wl

# name -> (n_g, n_bf, n_orb, n_occ, n_mu, n_types, n_terms)
SIZES = {
    "h6_chain": (4800, 24, 24, 3, 96, 1, 0),
    "h50_chain": (100000, 550, 400, 25, 2000, 1, 0),
    "h20_chain": (40000, 160, 160, 10, 800, 1, 28),
    "benzene": (271800, 1200, 1200, 21, 8000, 2, 10),
}


@pytest.mark.parametrize("name", sorted(SIZES))
def test_workload_sizes_weights_and_orthonormal_orbitals(name):
    w = wl.CONFIGS[name]()
    n_g, n_bf, n_orb, n_occ, n_mu, n_types, n_terms = SIZES[name]
    assert w.grid_xyz.shape == (n_g, 3) and w.grid_w.shape == (n_g,)
    assert w.basis.center.shape[0] == n_bf and w.mo_coef.shape == (n_bf, n_orb)
    assert (w.n_occ, w.n_mu) == (n_occ, n_mu)
    assert (w.jastrow.n_types, w.jastrow.n_terms) == (n_types, n_terms)
    assert np.all(np.isfinite(w.grid_xyz)) and np.all(w.grid_w > 0)
    # distinct points never coincide: the tensor-core radial generator
    # identifies the self pair by its exactly-zero difference vector
    nn, _ = cKDTree(w.grid_xyz).query(w.grid_xyz, k=2)
    assert nn[:, 1].min() > 1e-6
    S = wl.ao_overlap_fast(w.basis)
    assert np.allclose(np.diag(S), 1.0, rtol=0, atol=1e-12)
    C = w.mo_coef
    assert np.max(np.abs(C.T @ S @ C - np.eye(n_orb))) < 1e-5


def test_perturbed_chain_family():
    spacings = []
    for k in range(3):
        w = wl.h30_chain_perturbed(k)
        assert w.n_g == 60000 and w.n_orb == 240 and w.n_mu == 1200
        z = np.sort(w.xyz[:, 2])
        spacings.append(np.mean(np.diff(z)))
        assert np.all(np.abs(np.diff(z) - spacings[-1]) < 0.11)
    assert all(1.6 - 0.01 < s < 2.2 + 0.01 for s in spacings)
    assert len(set(np.round(spacings, 6))) == 3
