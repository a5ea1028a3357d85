"""ISDF Jastrow kernels u^(1),c and u^(3) (Eqs. K1-isdf, K3-isdf) -- oracle.

TEST INFRASTRUCTURE (FP64 numpy, grid batches).

  u1^c[mu, nu] = sum_{g,g'} w_g w_g' xi~^c_mu(g) xi_nu(g') K_c(g, g')
  u3[mu, nu]   = sum_{g,g'} w_g w_g' xi_mu(g)  xi_nu(g') K_sq(g, g')
evaluated in two stages as the paper's intermediates suggest:
  calG^c[nu, g] = sum_g' w_g' xi_nu(g') K_c(g, g')     (calG of Sec. III.B)
  T[nu, g]      = sum_g' w_g' xi_nu(g') K_sq(g, g')
  u1^c = (w xi~^c) calG^c^T,  u3 = (w xi) T^T.
Output W[4][n_mu][n_mu] in the order (x, y, z, sq).
"""
from __future__ import annotations

import numpy as np

from . import jastrow as J


def stage1(grid, w, xi, jas, g_rows=None, batch: int = 512, cols=None):
    """calG [4][n_nu][len(g_rows)] for the rows g in ``g_rows`` (default all);
    ``cols`` restricts nu."""
    n_g = grid.shape[0]
    rows = np.arange(n_g) if g_rows is None else np.asarray(g_rows)
    wxi = (xi if cols is None else xi[cols]) * w[None, :]
    out = np.zeros((4, wxi.shape[0], rows.shape[0]))
    allg = np.arange(n_g)
    for b0 in range(0, rows.shape[0], batch):
        r = rows[b0:b0 + batch]
        K = J.kernels(grid[r], grid, jas, r, allg)          # [4, nb, n_g]
        for c in range(4):
            out[c][:, b0:b0 + batch] = wxi @ K[c].T
    return out


def stage2(w, xi, xit, calG, g_rows=None):
    """W [4][n_mu][n_nu] from calG over the rows in g_rows."""
    rows = slice(None) if g_rows is None else g_rows
    W = np.empty((4, xi.shape[0], calG.shape[1]))
    for c in range(3):
        W[c] = (xit[c][:, rows] * w[None, rows]) @ calG[c].T
    W[3] = (xi[:, rows] * w[None, rows]) @ calG[3].T
    return W


def build(grid, w, xi, xit, jas, batch: int = 512):
    """W [4][n_mu][n_mu] of Eqs. K1-isdf and K3-isdf (channels x, y, z, sq) and
    calG, by stage1 then stage2."""
    calG = stage1(grid, w, xi, jas, batch=batch)
    return stage2(w, xi, xit, calG), calG


def brute_force(grid, w, xi, xit, jas):
    """Direct quadruple sum, pure loops over (g, g'); tiny inputs only."""
    n_g = grid.shape[0]
    n_mu = xi.shape[0]
    W = np.zeros((4, n_mu, n_mu))
    K = J.kernels(grid, grid, jas, np.arange(n_g), np.arange(n_g))
    for g in range(n_g):
        for h in range(n_g):
            ww = w[g] * w[h]
            for c in range(3):
                W[c] += ww * K[c, g, h] * np.outer(xit[c][:, g], xi[:, h])
            W[3] += ww * K[3, g, h] * np.outer(xi[:, g], xi[:, h])
    return W


def stage1_bounded(grid, w, xi, jas, g_rows, batch: int = 128):
    """calG of ``stage1`` for the rows in g_rows together with the normwise
    bound sum_g' |w_g' xi_nu(g')| |K_c(g, g')| of each of its sums (the scale
    of a dot product's rounding error); both [4][n_nu][len(g_rows)]."""
    n_g = grid.shape[0]
    rows = np.asarray(g_rows)
    wxi = xi * w[None, :]
    awxi = np.abs(wxi)
    out = np.zeros((4, wxi.shape[0], rows.shape[0]))
    bound = np.zeros_like(out)
    allg = np.arange(n_g)
    for b0 in range(0, rows.shape[0], batch):
        r = rows[b0:b0 + batch]
        K = J.kernels(grid[r], grid, jas, r, allg)
        for c in range(4):
            out[c][:, b0:b0 + batch] = wxi @ K[c].T
            bound[c][:, b0:b0 + batch] = awxi @ np.abs(K[c]).T
    return out, bound
