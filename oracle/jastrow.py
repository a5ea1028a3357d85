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

One-body nuclear-cusp term (Eq. tau-def): u = u2 + [chi(r_i) + chi(r_j)]/(N-1),
so that sum_{i<j} u = sum_i chi(r_i) + sum_{i<j} u2 for N electrons, and each
ordered pair carries grad chi(r_i)/(N-1) in its electron-1 gradient.  The paper
takes chi from a cited work without stating it; the reading used here is
   chi(r) = sum_I a_t r_iI / (1 + beta_t r_iI),   t = type(I),
whose slope at nucleus I is a_t (a_t = -Z_t imposes the electron-nucleus
cusp) and which tends to a_t/beta_t far away.  chi is off when the object
has no chi_a or all chi_a are zero.
"""
from __future__ import annotations

import numpy as np


def _unit(dv: np.ndarray, r: np.ndarray) -> np.ndarray:
    with np.errstate(invalid="ignore", divide="ignore"):
        u = dv / r[..., None]
    return np.where(r[..., None] > 0, u, 0.0)


def chi_on(jas) -> bool:
    a = getattr(jas, "chi_a", None)
    return a is not None and bool(np.any(np.asarray(a) != 0.0))


def chi_value(r: np.ndarray, jas) -> np.ndarray:
    """chi(r) = sum_I a_t r_I / (1 + beta_t r_I) at points r [n, 3] -> [n]."""
    out = np.zeros(r.shape[0])
    for I in range(jas.n_nuc):
        t = jas.nuc_type[I]
        rI = np.linalg.norm(r - jas.nuc_xyz[I], axis=1)
        out += jas.chi_a[t] * rI / (1.0 + jas.chi_b[t] * rI)
    return out


def chi_grad(r: np.ndarray, jas) -> np.ndarray:
    """grad chi at points r [n, 3] -> [3, n]: a_t / (1 + beta_t r_I)^2 e_I,
    with a zero direction on a nucleus."""
    out = np.zeros((3, r.shape[0]))
    for I in range(jas.n_nuc):
        t = jas.nuc_type[I]
        dv = r - jas.nuc_xyz[I]
        rI = np.linalg.norm(dv, axis=1)
        s = jas.chi_a[t] / (1.0 + jas.chi_b[t] * rI) ** 2
        out += (s[:, None] * _unit(dv, rI)).T
    return out


def u_value(ri: np.ndarray, rj: np.ndarray, jas) -> np.ndarray:
    """u(r_i, r_j) of Eqs. bh-scaled and bh-u (plus the cusp term and the
    one-body term of Eq. tau-def) for all pairs, [n, m]."""
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
    if chi_on(jas):
        u += (chi_value(ri, jas)[:, None] + chi_value(rj, jas)[None, :]) / (jas.n_elec - 1)
    return u


def grad1_u(ri: np.ndarray, rj: np.ndarray, jas) -> np.ndarray:
    """Analytic d u(r_i, r_j) / d r_i of Eqs. bh-scaled and bh-u (and of the
    one-body term of Eq. tau-def), [3, n, m]."""
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
    if chi_on(jas):
        g += chi_grad(ri, jas)[:, :, None] / (jas.n_elec - 1)
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
