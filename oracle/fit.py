"""Least-squares ISDF fit of the auxiliary densities (Eq. isdf-rho) -- oracle.

TEST INFRASTRUCTURE (FP64 numpy/scipy).

Given pivots r_mu:
  G[mu, g]    = sum_p phi_p(r_mu) phi_p(r_g)
  scalar:     Gram = G_PP o G_PP,        RHS[mu, g] = G[mu, g]^2
  gradient c: Gram = (dG^c)_PP o G_PP,   RHS[mu, g] = dG^c[mu, g] G[mu, g]
              with dG^c[mu, g] = sum_p d_c phi_p(r_mu) d_c phi_p(r_g)
  xi = Gram^{-1} RHS by Cholesky (Sec. II.D normal equations).
Reading of the adaptive Tikhonov shift (Sec. IV.B): try lambda = 0; on
failure lambda = 1e-14 max(diag), times 10 per retry, at most 8 retries.
Weights do not enter xi (each grid column is solved on its own).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def cholesky_with_jitter(A: np.ndarray, max_tries: int = 8):
    """Lower Cholesky factor of A + lambda I and the lambda used: the adaptive
    Tikhonov retry of Sec. IV.B with the schedule read in the module docstring."""
    try:
        return sla.cholesky(A, lower=True), 0.0
    except np.linalg.LinAlgError:
        pass
    lam = 1e-14 * float(np.max(np.diag(A)))
    for _ in range(max_tries):
        try:
            return sla.cholesky(A + lam * np.eye(A.shape[0]), lower=True), lam
        except np.linalg.LinAlgError:
            lam *= 10.0
    raise np.linalg.LinAlgError("Gram matrix not positive definite after jitter")


def grams(phi, dphi, piv):
    """The four normal-equation matrices [4][n_mu][n_mu] (scalar, x, y, z) of
    the least-squares fits of Sec. II.D."""
    phiP = phi[:, piv].T
    GPP = phiP @ phiP.T
    out = [GPP * GPP]
    for c in range(3):
        dP = dphi[c][:, piv].T
        out.append((dP @ dP.T) * GPP)
    return np.stack(out)


def rhs(phi, dphi, piv, g0=0, g1=None):
    """Right-hand sides [4][n_mu][g1-g0] of the normal equations of Sec. II.D."""
    g1 = phi.shape[1] if g1 is None else g1
    phiP = phi[:, piv].T
    G = phiP @ phi[:, g0:g1]
    out = [G * G]
    for c in range(3):
        dP = dphi[c][:, piv].T
        out.append((dP @ dphi[c][:, g0:g1]) * G)
    return np.stack(out)


def fit(phi, dphi, piv, channels=(0, 1, 2, 3)):
    """xi [n_mu][n_g] and xi~ [3][n_mu][n_g] of Eq. isdf-rho and its gradient
    analogue (Sec. II.D normal equations), plus the jitter per channel."""
    Gm = grams(phi, dphi, piv)
    B = rhs(phi, dphi, piv)
    xis = np.zeros_like(B)
    lams = np.zeros(4)
    for c in channels:
        L, lam = cholesky_with_jitter(Gm[c])
        lams[c] = lam
        xis[c] = sla.cho_solve((L, True), B[c])
    return xis[0], xis[1:], lams


def fit_residual(phi, w, piv, xi):
    """Weighted scalar-channel fit residual per point,
    w_g^2 [ (sum_p phi_p^2)^2 - sum_mu xi_mu(g) G[mu, g]^2 ]  (the squared
    Frobenius residual of Eq. isdf-rho on the weight-scaled grid)."""
    G = phi[:, piv].T @ phi
    dens = np.sum(phi * phi, axis=0)
    return (w * w) * (dens * dens - np.sum(xi * G * G, axis=0))
