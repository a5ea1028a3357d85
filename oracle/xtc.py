"""xTC density contraction of the three-body term (Sec. III.B) -- oracle.

TEST INFRASTRUCTURE (FP64 numpy).

The reference density matrix is the closed-shell HF projector onto the first
n_occ orbitals, gamma^u_t = delta_ut [t < n_occ] (idempotent in the MO basis),
so the low-rank projector L_Q is the set of occupied unit vectors.

  C^p_q(mu)     = phi_p(r_mu) phi_q(r_mu)                    pivot tensor
  G_nu          = sum_{tu} C^t_u(nu) gamma^u_t
  L^u_{s nu}    = sum_t gamma^u_t C^t_s(nu)
  calG^c[mu, g] = sum_g' w_g' xi_mu(g') d_c u(g, g')         (from wbuild)
  w~_g   = w_g sum_l G_l xi_l(g)
  D4     = sum_g w~_g sum_c calG^c_mu calG^c_nu
  H_gc   = sum_l G_l calG^c_{l g};   V_{nu g} = sum_c H_gc calG^c_{nu g}
  D1     = sum_g w_g xi_mu(g) V_{nu g};   D = D4 + 2 D1          (Eq. delta-u-dx-kernels)
  X = X2 + X31 + X32 with Y, Z, L~, C^ as defined in the paper (dense form)
  or, in the low-rank projector form, with the occupied fields
     A^s_{a,g,c} = sum_nu C^a_s(nu) calG^c_{nu g},  rho~^s_a(g) = sum_nu C^a_s(nu) xi_nu(g)
  X_{qs mu} = sum_g w_g [ xi_mu(g) sum_{a,c} A^s_{a,c} A^q_{a,c}
                         + sum_c calG^c_{mu g} sum_a (rho~^s_a A^q_{a,c} + A^s_{a,c} rho~^q_a) ]
Packed output: row s(s+1)/2 + q holds X_{qs .} for q <= s.
"""
from __future__ import annotations

import numpy as np


def pivot_factors(phi, piv):
    """phi_p(r_mu) [n_mu][n_orb]: the orbital values at the pivots that form the
    pivot tensors C^p_q(r_mu) = phi_p(r_mu) phi_q(r_mu) of Eq. isdf-rho."""
    return np.ascontiguousarray(phi[:, piv].T)     # [n_mu][n_orb]


def g_nu(phiP, n_occ):
    """G_nu = sum_{tu} C^t_u(r_nu) gamma^u_t of Sec. III.B with gamma the
    projector on the first n_occ orbitals: sum_{i < n_occ} phi_i(r_nu)^2."""
    return np.sum(phiP[:, :n_occ] ** 2, axis=1)


def d_kernels(w, xi, calG, Gnu):
    """D4, D1, D = D4 + 2 D1 from calG [>=3][n_mu][n_g]."""
    wt = w * (Gnu @ xi)
    D4 = np.zeros((xi.shape[0], xi.shape[0]))
    V = np.zeros_like(xi)
    for c in range(3):
        D4 += (calG[c] * wt[None, :]) @ calG[c].T
        H = Gnu @ calG[c]
        V += H[None, :] * calG[c]
    D1 = (xi * w[None, :]) @ V.T
    return D4, D1, D4 + 2.0 * D1


def x_dense(w, xi, calG, phiP, n_occ):
    """X [n_orb][n_orb][n_mu] via the paper's Y, Z, L~, C^ intermediates
    (sum over all u with gamma inside L).  Small inputs only."""
    n_mu, n_orb = phiP.shape
    gamma = np.zeros((n_orb, n_orb))
    gamma[np.arange(n_occ), np.arange(n_occ)] = 1.0
    C = phiP[:, :, None] * phiP[:, None, :]              # [nu, t, s]
    L = np.einsum("ut,nts->usn", gamma, C)               # L^u_{s nu}
    Y = np.einsum("usn,cng->usgc", L, calG[:3])
    Z = np.einsum("nqu,cng->qugc", C, calG[:3])
    Lt = np.einsum("usn,ng->usg", L, xi)
    Ch = np.einsum("nqu,ng->qug", C, xi)
    wxi = xi * w[None, :]
    X2 = np.einsum("mg,usgc,qugc->qsm", wxi, Y, Z)
    wG = calG[:3] * w[None, None, :]
    X31 = np.einsum("cmg,usg,qugc->qsm", wG, Lt, Z)
    X32 = np.einsum("cmg,usgc,qug->qsm", wG, Y, Ch)
    return X2, X31 + X32


def x_projector(w, xi, calG, phiP, n_occ):
    """X [n_orb][n_orb][n_mu] in the low-rank projector form."""
    occ = phiP[:, :n_occ]
    Cao = occ[:, :, None] * phiP[:, None, :]             # [nu, a, s]
    A = np.einsum("nas,cng->ascg", Cao, calG[:3])        # [a, s, c, g]
    rt = np.einsum("nas,ng->asg", Cao, xi)               # [a, s, g]
    wxi = xi * w[None, :]
    AA = np.einsum("ascg,aqcg->qsg", A, A)
    X = np.einsum("mg,qsg->qsm", wxi, AA)
    wG = calG[:3] * w[None, None, :]
    M = np.einsum("asg,aqcg->qscg", rt, A) + np.einsum("ascg,aqg->qscg", A, rt)
    X += np.einsum("cmg,qscg->qsm", wG, M)
    return X


def pack_upper(X):
    """[n_orb][n_orb][n_mu] -> [n_orb (n_orb+1)/2][n_mu], row s(s+1)/2 + q."""
    n = X.shape[0]
    rows = []
    for s in range(n):
        for q in range(s + 1):
            rows.append(X[q, s])
    return np.array(rows)
