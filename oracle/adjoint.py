"""Adjoint of the Jastrow kernels with respect to the correlator parameters --
oracle (not in the paper).

TEST INFRASTRUCTURE (FP64 numpy, analytic derivatives written from the
Boys-Handy form of Eqs. bh-scaled / bh-u).

Parameters theta = (d, b_0 .. b_{T-1}, c[0][0] .. c[T-1][K-1]) (type-major).
For a seed Wbar = {Wbar^x, Wbar^y, Wbar^z, Wbar^sq} the scalar
    L(theta) = sum_c <Wbar^c, W^c(theta)>
with W from Eqs. K1-isdf / K3-isdf has the gradient
    dL/dtheta_j = sum_{g,g'} sum_{c<3} (M^c(g,g') + 2 M^sq(g,g') K_c(g,g')) d K_c(g,g') / d theta_j
    M^c(g,g')   = w_g w_g' [xi~^c^T Wbar^c xi]_{g g'}      (c = x, y, z)
    M^sq(g,g')  = w_g w_g' [xi^T Wbar^sq xi]_{g g'}
because K_sq = sum_c K_c^2.  The self pair contributes nothing (K = 0 there).

grad_1 u = cE dE/dr e_ij + sum_I cA_I grad A_iI with
    cE   = cusp/(2d) + sum_I sum_k c_k [A_i^m A_j^n + A_j^m A_i^n] o E^(o-1)
    cA_I = sum_k c_k [m A_i^(m-1) A_j^n + n A_j^m A_i^(n-1)] E^o
and every derivative below is the chain rule applied to these factors.
"""
from __future__ import annotations

import numpy as np

from . import jastrow as J


def n_params(jas) -> int:
    """Number of parameters theta = (d, b per type, c per type and term) of
    the correlator of Eqs. bh-scaled and bh-u."""
    return 1 + jas.n_types + jas.n_types * jas.n_terms


def get_theta(jas) -> np.ndarray:
    """theta = (d, b_0 .. b_{T-1}, c[type][term] row-major) of Eqs. bh-scaled, bh-u."""
    return np.concatenate([[jas.d], np.asarray(jas.b, float), np.asarray(jas.coef, float).ravel()])


def set_theta(jas, theta):
    """A copy of the correlator with the parameters theta (order of get_theta)."""
    import copy
    j2 = copy.deepcopy(jas)
    j2.d = float(theta[0])
    T = jas.n_types
    j2.b = np.array(theta[1:1 + T], float)
    j2.coef = np.array(theta[1 + T:], float).reshape(T, jas.n_terms)
    return j2


def _pw(x, n):
    return x ** n if n >= 0 else np.zeros_like(x)


def dgrad_dtheta(ri, rj, jas):
    """d(grad_1 u)/d theta for all pairs: [n_params, 3, n, m]."""
    T, Kt = jas.n_types, jas.n_terms
    P = n_params(jas)
    dv = ri[:, None, :] - rj[None, :, :]
    r = np.sqrt(np.sum(dv * dv, axis=2))
    with np.errstate(invalid="ignore", divide="ignore"):
        eij = np.where(r[..., None] > 0, dv / r[..., None], 0.0)
    d = jas.d
    den = 1.0 + d * r
    E = d * r / den
    dEdr = d / den ** 2
    E_d = r / den ** 2                 # dE/dd
    dEdr_d = (1.0 - d * r) / den ** 3  # d(dE/dr)/dd
    out = np.zeros((P, 3) + r.shape)
    cE = np.zeros_like(r) + (0.5 / d if jas.cusp else 0.0)
    cE_d = np.zeros_like(r) + (-0.5 / d ** 2 if jas.cusp else 0.0)
    cE_b = np.zeros((T,) + r.shape)
    cE_c = np.zeros((T, Kt) + r.shape)
    gA_tot_d = np.zeros((3,) + r.shape)        # sum_I dcA_I/dd gradA
    gA_b = np.zeros((T, 3) + r.shape)          # sum_{I in t} d(cA_I gradA)/db_t
    gA_c = np.zeros((T, Kt, 3) + r.shape)      # sum_{I in t} dcA_I/dc gradA
    for I in range(jas.n_nuc):
        t = jas.nuc_type[I]
        b = jas.b[t]
        dvi = ri - jas.nuc_xyz[I]
        riI = np.linalg.norm(dvi, axis=1)
        rjI = np.linalg.norm(rj - jas.nuc_xyz[I], axis=1)
        with np.errstate(invalid="ignore", divide="ignore"):
            eI = np.where(riI[:, None] > 0, dvi / riI[:, None], 0.0)
        dni, dnj = 1.0 + b * riI, 1.0 + b * rjI
        Ai = (b * riI / dni)[:, None]
        Aj = (b * rjI / dnj)[None, :]
        Ai_b = (riI / dni ** 2)[:, None]
        Aj_b = (rjI / dnj ** 2)[None, :]
        gA = (b / dni ** 2)[:, None] * eI          # [n, 3]
        gA_bb = ((1.0 - b * riI) / dni ** 3)[:, None] * eI
        cA = np.zeros_like(r)
        cA_d = np.zeros_like(r)
        cA_b = np.zeros_like(r)
        for k in range(Kt):
            m, n, o = (int(x) for x in jas.mno[k])
            c = jas.coef[t, k]
            S = Ai ** m * Aj ** n + Aj ** m * Ai ** n
            S_b = (m * _pw(Ai, m - 1) * Aj ** n * Ai_b + n * Ai ** m * _pw(Aj, n - 1) * Aj_b
                   + m * _pw(Aj, m - 1) * Ai ** n * Aj_b + n * Aj ** m * _pw(Ai, n - 1) * Ai_b)
            Da = m * _pw(Ai, m - 1) * Aj ** n + n * Aj ** m * _pw(Ai, n - 1)
            Da_b = (m * (m - 1) * _pw(Ai, m - 2) * Aj ** n * Ai_b
                    + m * n * _pw(Ai, m - 1) * _pw(Aj, n - 1) * Aj_b
                    + n * m * _pw(Aj, m - 1) * _pw(Ai, n - 1) * Aj_b
                    + n * (n - 1) * Aj ** m * _pw(Ai, n - 2) * Ai_b)
            Eo = E ** o
            Eo_d = o * _pw(E, o - 1) * E_d
            # cE pieces
            if o > 0:
                Eo1 = E ** (o - 1)
                Eo1_d = (o - 1) * _pw(E, o - 2) * E_d
                cE += c * S * o * Eo1
                cE_d += c * S * o * Eo1_d
                cE_b[t] += c * S_b * o * Eo1
                cE_c[t, k] += S * o * Eo1
            # cA pieces
            cA += c * Da * Eo
            cA_d += c * Da * Eo_d
            cA_b += c * Da_b * Eo
            for ax in range(3):
                gA_c[t, k, ax] += Da * Eo * gA[:, ax][:, None]
        for ax in range(3):
            gA_tot_d[ax] += cA_d * gA[:, ax][:, None]
            gA_b[t, ax] += cA_b * gA[:, ax][:, None] + cA * gA_bb[:, ax][:, None]
    for ax in range(3):
        e = eij[:, :, ax]
        out[0, ax] = (cE_d * dEdr + cE * dEdr_d) * e + gA_tot_d[ax]
        for t in range(T):
            out[1 + t, ax] = cE_b[t] * dEdr * e + gA_b[t, ax]
            for k in range(Kt):
                out[1 + T + t * Kt + k, ax] = cE_c[t, k] * dEdr * e + gA_c[t, k, ax]
    return out


def loss(grid, w, xi, xit, jas, Wbar):
    """L(theta) = sum_c <Wbar^c, W^c> with W from the oracle's W build."""
    from . import wbuild
    W, _ = wbuild.build(grid, w, xi, xit, jas)
    return float(np.sum(Wbar * W))


def grad(grid, w, xi, xit, jas, Wbar, batch: int = 256):
    """dL/dtheta by the formula in the module docstring (FP64)."""
    n_g = grid.shape[0]
    P = n_params(jas)
    wxi = xi * w[None, :]
    # Bhat^c = Wbar^c (w xi) : [4][n_mu][n_g]
    Bh = np.stack([Wbar[c] @ wxi for c in range(4)])
    out = np.zeros(P)
    allg = np.arange(n_g)
    for g0 in range(0, n_g, batch):
        rows = np.arange(g0, min(g0 + batch, n_g))
        K = J.kernels(grid[rows], grid, jas, rows, allg)      # [4, nb, n_g]
        dK = dgrad_dtheta(grid[rows], grid, jas)              # [P, 3, nb, n_g]
        same = rows[:, None] == allg[None, :]
        dK[:, :, same] = 0.0
        Msq = (xi[:, rows] * w[rows][None, :]).T @ Bh[3]      # [nb, n_g]
        for c in range(3):
            Mc = (xit[c][:, rows] * w[rows][None, :]).T @ Bh[c]
            coef = Mc + 2.0 * Msq * K[c]
            out += np.einsum("gh,pgh->p", coef, dK[:, c])
    return out
