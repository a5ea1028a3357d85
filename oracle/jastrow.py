"""Boys-Handy correlator and its electron-1 gradient -- oracle.

TEST INFRASTRUCTURE (FP64 numpy).

Scaled distances (Eq. bh-scaled):  A_iI = b_I r_iI / (1 + b_I r_iI),
                                   E_ij = d r_ij / (1 + d r_ij).
Correlator (Eq. bh-u):
   u(i,j) = sum_I sum_k c_k^I [A_iI^m A_jI^n + A_jI^m A_iI^n] E_ij^o
          + [cusp]  E_ij / (2 d)
The cusp line is the (m,n,o) = (0,0,1) term with prefactor 1/(4 N_nuc d)
summed over the N_nuc centres; its slope du/dr_ij at r_ij -> 0 is 1/2
(opposite-spin Kato condition, Sec. II.B).

The kernels that enter u^(1) and u^(3) (Eqs. K1-isdf, K3-isdf) are
   K_c(g,g')  = d u(r_g, r_g') / d r_{g,c}      c = x, y, z
   K_sq(g,g') = sum_c K_c(g,g')^2
Reading: the self pair g = g' has no defined gradient direction; K_c and
K_sq are set to 0 there (mask by index).  A point on a nucleus gets a zero
direction for that nucleus.
"""
from __future__ import annotations

import numpy as np


def _unit(dv: np.ndarray, r: np.ndarray) -> np.ndarray:
    with np.errstate(invalid="ignore", divide="ignore"):
        u = dv / r[..., None]
    return np.where(r[..., None] > 0, u, 0.0)


def u_value(ri: np.ndarray, rj: np.ndarray, jas) -> np.ndarray:
    """u(r_i, r_j) of Eqs. bh-scaled and bh-u (plus the cusp term) for all pairs, [n, m]."""
    dv = ri[:, None, :] - rj[None, :, :]
    r = np.sqrt(np.sum(dv * dv, axis=2))
    E = jas.d * r / (1.0 + jas.d * r)
    u = np.zeros_like(r)
    if jas.cusp:
        u += E / (2.0 * jas.d)
    for I in range(jas.n_nuc):
        t = jas.nuc_type[I]
        bI = jas.b[t]
        riI = np.linalg.norm(ri - jas.nuc_xyz[I], axis=1)
        rjI = np.linalg.norm(rj - jas.nuc_xyz[I], axis=1)
        Ai = (bI * riI / (1.0 + bI * riI))[:, None]
        Aj = (bI * rjI / (1.0 + bI * rjI))[None, :]
        for k in range(jas.n_terms):
            m, n, o = (int(x) for x in jas.mno[k])
            c = jas.coef[t, k]
            u += c * (Ai ** m * Aj ** n + Aj ** m * Ai ** n) * E ** o
    return u


def grad1_u(ri: np.ndarray, rj: np.ndarray, jas) -> np.ndarray:
    """Analytic d u(r_i, r_j) / d r_i of Eqs. bh-scaled and bh-u, [3, n, m]."""
    dv = ri[:, None, :] - rj[None, :, :]
    r = np.sqrt(np.sum(dv * dv, axis=2))
    d = jas.d
    E = d * r / (1.0 + d * r)
    dEdr = d / (1.0 + d * r) ** 2
    eij = _unit(dv, r)                                      # [n, m, 3]
    # scalar coefficient multiplying grad E = dEdr * e_ij
    cE = np.zeros_like(r)
    if jas.cusp:
        cE += 1.0 / (2.0 * d)
    g = np.zeros((3,) + r.shape)
    for I in range(jas.n_nuc):
        t = jas.nuc_type[I]
        bI = jas.b[t]
        dvi = ri - jas.nuc_xyz[I]
        riI = np.linalg.norm(dvi, axis=1)
        rjI = np.linalg.norm(rj - jas.nuc_xyz[I], axis=1)
        Ai = (bI * riI / (1.0 + bI * riI))[:, None]
        Aj = (bI * rjI / (1.0 + bI * rjI))[None, :]
        dAi = (bI / (1.0 + bI * riI) ** 2)[:, None] * _unit(dvi, riI)   # [n, 3]
        cA = np.zeros_like(r)   # coefficient multiplying grad A_iI
        for k in range(jas.n_terms):
            m, n, o = (int(x) for x in jas.mno[k])
            c = jas.coef[t, k]
            Eo = E ** o
            da = np.zeros_like(r)
            if m > 0:
                da = da + m * Ai ** (m - 1) * Aj ** n
            if n > 0:
                da = da + n * Aj ** m * Ai ** (n - 1)
            cA += c * da * Eo
            if o > 0:
                cE += c * (Ai ** m * Aj ** n + Aj ** m * Ai ** n) * o * E ** (o - 1)
        for ax in range(3):
            g[ax] += cA * dAi[:, ax][:, None]
    for ax in range(3):
        g[ax] += cE * dEdr * eij[:, :, ax]
    return g


def kernels(ri: np.ndarray, rj: np.ndarray, jas, gi: np.ndarray = None,
            gj: np.ndarray = None) -> np.ndarray:
    """[K_x, K_y, K_z, K_sq] of Eqs. K1-isdf and K3-isdf for all pairs,
    [4, n, m].  ``gi``/``gj`` are the grid indices of the two point sets;
    pairs with gi == gj are zeroed."""
    g = grad1_u(ri, rj, jas)
    out = np.empty((4,) + g.shape[1:])
    out[:3] = g
    out[3] = np.sum(g * g, axis=0)
    if gi is not None and gj is not None:
        same = gi[:, None] == gj[None, :]
        out[:, same] = 0.0
    return out
