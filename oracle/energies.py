"""Four-index K and Delta U from the ISDF factors and the closed-shell test
energies -- oracle.

TEST INFRASTRUCTURE (FP64 numpy).

  K1^{pq}_{rs} = sum_{mu nu} sum_c u1^c_{mu nu} phi_p(mu) d_c phi_r(mu) phi_q(nu) phi_s(nu)
  K3^{pq}_{rs} = sum_{mu nu} u3_{mu nu} C^p_r(mu) C^q_s(nu)                 (Eqs. K1-isdf, K3-isdf)
  K = 1/2 P12 [K1 - K1swap + K3],  K1swap^{pq}_{rs} = K1^{rs}_{pq},
  P12 T^{pq}_{rs} = T^{pq}_{rs} + T^{qp}_{sr}                               (Eq. K-recombine-final)
  DeltaU = -P12 [ sum C^p_r(mu) D_{mu nu} C^q_s(nu) - sum_mu C^p_r(mu) X_{qs mu} ]
  Delta h_pq = -1/2 sum_o (2 DeltaU^{po}_{qo} - DeltaU^{po}_{oq})          (Eq. xtc-deltah)
  f^xTC_pq = Delta h_pq + sum_i (2 W^{pi}_{qi} - W^{pi}_{iq}),  W = -K + DeltaU  (Eq. xtc-fock)
  E0 = -2/3 sum_i Delta h_ii   (nuclear repulsion omitted)                  (Eq. xtc-const)
Closed-shell test functionals (reading of "TC energy"):
  E_K = sum_{ij occ} (2 K^{ij}_{ij} - K^{ij}_{ji}),  E_dU likewise with DeltaU.
"""
from __future__ import annotations

import numpy as np


def k_tensor(W, phiP, dphiP, idx):
    """K^{pq}_{rs} for p, q, r, s in ``idx`` -> [n][n][n][n] (p, q, r, s), from
    u^(1) and u^(3) (Eqs. K1-isdf, K3-isdf) recombined by Eq. K-recombine-final."""
    P = phiP[:, idx]
    dP = [d[:, idx] for d in dphiP]
    Cs = P[:, :, None] * P[:, None, :]                     # [mu, q, s]
    K1 = np.zeros((len(idx),) * 4)
    for c in range(3):
        Ct = P[:, :, None] * dP[c][:, None, :]             # [mu, p, r]
        K1 += np.einsum("mpr,mn,nqs->pqrs", Ct, W[c], Cs)
    K3 = np.einsum("mpr,mn,nqs->pqrs", Cs, W[3], Cs)
    K1swap = np.transpose(K1, (2, 3, 0, 1))                 # K1^{rs}_{pq}
    T = K1 - K1swap + K3
    return 0.5 * (T + np.transpose(T, (1, 0, 3, 2)))


def du_tensor(D, X, phiP, idx):
    """DeltaU^{pq}_{rs} for p, q, r, s in idx by the final assembly of Sec. III.B
    (Eq. deltaU-four with the D and X kernels).  X is [n_orb][n_orb][n_mu]."""
    P = phiP[:, idx]
    Cs = P[:, :, None] * P[:, None, :]                     # [mu, p, r]
    T1 = np.einsum("mpr,mn,nqs->pqrs", Cs, D, Cs)
    Xs = X[np.ix_(idx, idx)]                               # [q, s, mu]
    T2 = np.einsum("mpr,qsm->pqrs", Cs, Xs)
    T = T1 - T2
    return -(T + np.transpose(T, (1, 0, 3, 2)))


def closed_shell(T):
    """sum_{ij} (2 T^{ij}_{ij} - T^{ij}_{ji}) over the given (occupied) block: the
    closed-shell expectation value read as the test energy (Coulomb weight 2 and
    exchange, as in Eq. xtc-fock)."""
    n = T.shape[0]
    i = np.arange(n)
    coul = T[i[:, None], i[None, :], i[:, None], i[None, :]]
    exch = T[i[:, None], i[None, :], i[None, :], i[:, None]]
    return float(np.sum(2.0 * coul - exch))


def delta_h_occ(dU):
    """Delta h_ii for i in the block (the block is the occupied space), Eq. xtc-deltah."""
    n = dU.shape[0]
    out = np.zeros(n)
    for i in range(n):
        out[i] = -0.5 * sum(2.0 * dU[i, o, i, o] - dU[i, o, o, i] for o in range(n))
    return out


def energies(W, D, X, phiP, dphiP, n_occ):
    """E_K and E_dU (closed_shell of K and DeltaU on the occupied block) and
    E0 = -2/3 sum_i Delta h_ii (Eq. xtc-const, without nuclear repulsion)."""
    occ = np.arange(n_occ)
    K = k_tensor(W, phiP, dphiP, occ)
    dU = du_tensor(D, X, phiP, occ)
    dh = delta_h_occ(dU)
    return {"E_K": closed_shell(K), "E_dU": closed_shell(dU),
            "E0": -2.0 / 3.0 * float(np.sum(dh))}


def delta_h(dU, occ):
    """Delta h_pq of Eq. xtc-deltah for every p, q: dU is the full four-index
    DeltaU [n][n][n][n] (index order p, q, r, s of DeltaU^{pq}_{rs}) and occ the
    occupied orbital indices."""
    return -0.5 * sum(2.0 * dU[:, o, :, o] - dU[:, o, o, :] for o in occ)


def fock_xtc(K, dU, occ):
    """f^xTC_pq of Eq. xtc-fock for every p, q: Delta h plus the closed-shell
    Coulomb (weight 2) and exchange contractions of W = -K + DeltaU over the
    occupied orbitals.  Not symmetrised (K and DeltaU are non-Hermitian)."""
    Wt = -K + dU
    return delta_h(dU, occ) + sum(2.0 * Wt[:, i, :, i] - Wt[:, i, i, :] for i in occ)


def e0_xtc(dh, occ):
    """E0 of Eq. xtc-const without the nuclear repulsion: -2/3 sum_i Delta h_ii."""
    return -2.0 / 3.0 * float(sum(dh[i, i] for i in occ))
