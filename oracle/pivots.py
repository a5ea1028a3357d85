"""Python front end of the order-exact pivot loop (Alg. 1, Sec. II.D).

TEST INFRASTRUCTURE.  See ``pivots.c`` for the arithmetic and the readings.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from . import build_oracle

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_oracle.build())
        f = _lib.oracle_pivots
        f.restype = ctypes.c_int
        P = ctypes.c_void_p
        f.argtypes = [P, P, P, ctypes.c_long, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                      ctypes.c_int, P, P, P, P, P, P, P, P, P, P]
        f = _lib.oracle_pivots_ranks
        f.restype = ctypes.c_int
        f.argtypes = [P, P, P, ctypes.c_long, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                      P, P, P, P, P, P]
    return _lib


@dataclasses.dataclass
class PivotResult:
    pivots: np.ndarray      # union, append order, int32
    piv_s: np.ndarray       # scalar-channel pivots
    piv_v: np.ndarray       # gradient-channel pivots
    d_s: np.ndarray         # final residual diagonals
    d_v: np.ndarray
    L_s: np.ndarray         # [n_s][n_g] Cholesky columns
    L_v: np.ndarray
    rank_exhausted: bool


MODES = {"fused": 0, "scalar": 1, "gradient": 2}


def select(phi: np.ndarray, dphi: np.ndarray, w: np.ndarray, n_mu: int,
           mode: str = "fused", cap: int = None, keep_L: bool = True) -> PivotResult:
    """Pivoted-Cholesky interpolation points (Alg. 1, its gradient branch and
    the pivot fusion of Sec. II.D, in the order-exact form of the C routine).
    phi [n_orb][n_g], dphi [3][n_orb][n_g], w [n_g]."""
    lib = _load()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    dphi = np.ascontiguousarray(dphi, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n_orb, n_g = phi.shape
    cap = n_mu if cap is None else cap
    pu = np.zeros(n_mu, np.int32)
    ps = np.zeros(cap, np.int32)
    pv = np.zeros(cap, np.int32)
    nu = ctypes.c_int(0)
    ns = ctypes.c_int(0)
    nv = ctypes.c_int(0)
    ds = np.zeros(n_g)
    dv = np.zeros(n_g)
    Ls = np.zeros((cap, n_g)) if keep_L else None
    Lv = np.zeros((cap, n_g)) if keep_L else None
    ptr = lambda a: None if a is None else a.ctypes.data
    rc = lib.oracle_pivots(ptr(phi), ptr(dphi), ptr(w), n_g, n_orb, n_mu, cap,
                           MODES[mode], ptr(pu), ctypes.byref(nu), ptr(ps),
                           ctypes.byref(ns), ptr(pv), ctypes.byref(nv), ptr(ds),
                           ptr(dv), ptr(Ls), ptr(Lv))
    return PivotResult(pivots=pu[:nu.value].copy(), piv_s=ps[:ns.value].copy(),
                       piv_v=pv[:nv.value].copy(), d_s=ds, d_v=dv,
                       L_s=None if Ls is None else Ls[:ns.value],
                       L_v=None if Lv is None else Lv[:nv.value],
                       rank_exhausted=bool(rc))


def select_ranks(phi: np.ndarray, dphi: np.ndarray, w: np.ndarray, n_phi: int,
                 n_grad: int) -> PivotResult:
    """The paper's pivot fusion (Sec. II.D): the scalar channel run to rank
    n_phi and the gradient channel to rank n_grad, each on its own (Alg. 1 and
    its gradient branch), then their union -- the scalar list followed by the
    gradient pivots not already in it.  L and d are not kept."""
    lib = _load()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    dphi = np.ascontiguousarray(dphi, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n_orb, n_g = phi.shape
    pu = np.zeros(max(n_phi + n_grad, 1), np.int32)
    ps = np.zeros(max(n_phi, 1), np.int32)
    pv = np.zeros(max(n_grad, 1), np.int32)
    nu, ns, nv = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    rc = lib.oracle_pivots_ranks(phi.ctypes.data, dphi.ctypes.data, w.ctypes.data, n_g, n_orb,
                                 n_phi, n_grad, pu.ctypes.data, ctypes.byref(nu),
                                 ps.ctypes.data, ctypes.byref(ns), pv.ctypes.data,
                                 ctypes.byref(nv))
    return PivotResult(pivots=pu[:nu.value].copy(), piv_s=ps[:ns.value].copy(),
                       piv_v=pv[:nv.value].copy(), d_s=None, d_v=None, L_s=None, L_v=None,
                       rank_exhausted=bool(rc))


def tie_margin(phi, dphi, w, piv_a, piv_b, channel: str):
    """Near-tie check for two pivot lists of one channel ("scalar" or
    "gradient") obtained from inputs equal up to rounding (e.g. orbitals
    evaluated on two machines).  Returns (j, gap): the first step j where the
    lists differ and the relative gap (d(a_j) - d(b_j)) / d(a_j) of this
    oracle's residual diagonal (Alg. 1) on (phi, dphi, w) just before step j,
    a_j being the point the oracle picks there.  (None, 0.0) when the lists
    agree over their common length."""
    n = min(len(piv_a), len(piv_b))
    diff = [j for j in range(n) if piv_a[j] != piv_b[j]]
    if not diff:
        return None, 0.0
    j = diff[0]
    st = select(phi, dphi, w, j, mode=channel, keep_L=False)   # the state after j steps
    d = st.d_s if channel == "scalar" else st.d_v
    a, b = int(piv_a[j]), int(piv_b[j])
    return j, float((d[a] - d[b]) / d[a])
