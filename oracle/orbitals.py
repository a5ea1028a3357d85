"""Orbitals and orbital gradients on the grid (Alg. 2 step 2) -- oracle.

TEST INFRASTRUCTURE: FP64 numpy, grid batches; no screening.

chi_f(r) = sum_k c_fk (x-X)^a (y-Y)^b (z-Z)^c exp(-alpha_fk |r-R|^2)
phi_p(r_g) = sum_f C[f, p] chi_f(r_g);  grad phi likewise with grad chi.
Layout: phi [n_orb][n_g], dphi [3][n_orb][n_g].
"""
from __future__ import annotations

import numpy as np


def eval_ao(basis, pts: np.ndarray):
    """Contracted Cartesian Gaussian values [n_bf, n] and analytic gradients
    [3, n_bf, n] at points [n, 3] (the basis functions of Alg. 2 step 2)."""
    n = pts.shape[0]
    nbf = basis.center.shape[0]
    val = np.zeros((nbf, n))
    grad = np.zeros((3, nbf, n))
    d = pts[None, :, :] - basis.center[:, None, :]          # [nbf, n, 3]
    r2 = np.sum(d * d, axis=2)                              # [nbf, n]
    pw = basis.powers
    for k in range(basis.exps.shape[1]):
        a = basis.exps[:, k][:, None]
        e = basis.coefs[:, k][:, None] * np.exp(-a * r2)     # [nbf, n]
        # polynomial part and its derivatives, axis by axis
        poly = np.ones((nbf, n))
        comp = []
        for ax in range(3):
            x = d[:, :, ax]
            p = pw[:, ax][:, None]
            xp = x ** p
            # d/dx [x^p exp(-a x^2)] / exp(...) = p x^(p-1) - 2 a x^(p+1)
            dxp = np.where(p > 0, p * x ** np.maximum(p - 1, 0), 0.0) - 2.0 * a * x ** (p + 1)
            comp.append((xp, dxp))
            poly = poly * xp
        val += poly * e
        for ax in range(3):
            other = np.ones((nbf, n))
            for bx in range(3):
                if bx != ax:
                    other = other * comp[bx][0]
            grad[ax] += comp[ax][1] * other * e
    return val, grad


def eval_orbitals(basis, mo_coef: np.ndarray, grid: np.ndarray, batch: int = 4096):
    """phi [n_orb][n_g] and dphi [3][n_orb][n_g] in FP64: the orbitals and their
    gradients on the grid (Alg. 2 step 2)."""
    n_g = grid.shape[0]
    n_orb = mo_coef.shape[1]
    phi = np.empty((n_orb, n_g))
    dphi = np.empty((3, n_orb, n_g))
    CT = mo_coef.T
    for g0 in range(0, n_g, batch):
        v, gr = eval_ao(basis, grid[g0:g0 + batch])
        phi[:, g0:g0 + batch] = CT @ v
        for c in range(3):
            dphi[c, :, g0:g0 + batch] = CT @ gr[c]
    return phi, dphi
