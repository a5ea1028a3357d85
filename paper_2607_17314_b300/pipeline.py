"""The ISDF-xTC kernel path, step by step (Alg. 2 steps 2-7) on one GPU.

  a1 orbitals -> a2 interpolation points -> a3 auxiliary fit -> a4 Jastrow
  kernels W = {u1x, u1y, u1z, u3} -> a5 xTC D (and X) -> a6 test energies

Inputs are plain arrays (a basis, MO coefficients, a grid with weights, a
Jastrow); every step runs in libisdftc.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, Optional

import numpy as np
import torch

from . import api


@dataclasses.dataclass
class Inputs:
    """Device-resident inputs of one pass: the basis, MO coefficients, grid and
    weights, N_mu, N_occ and the correlator struct."""
    center: torch.Tensor   # [n_bf][3]
    powers: torch.Tensor   # [n_bf][3] int32
    exps: torch.Tensor     # [n_bf][n_prim]
    coefs: torch.Tensor
    mo_coef: torch.Tensor  # [n_bf][n_orb]
    grid: torch.Tensor     # [n_g][3]
    w: torch.Tensor        # [n_g]
    n_mu: int
    n_occ: int
    jastrow: object        # isdf_jastrow struct

    @property
    def n_g(self):
        return self.grid.shape[0]


def upload(center, powers, exps, coefs, mo_coef, grid, w, n_mu, n_occ, jastrow,
           device="cuda", pin: bool = False) -> Inputs:
    """Copy host arrays to the device (from pinned host memory when ``pin``)."""
    def t(a, dt):
        x = torch.as_tensor(np.ascontiguousarray(a)).to(dt)
        if pin:
            x = x.pin_memory()
        return x.to(device, non_blocking=pin)
    return Inputs(t(center, torch.float64), t(powers, torch.int32), t(exps, torch.float64),
                  t(coefs, torch.float64), t(mo_coef, torch.float64), t(grid, torch.float64),
                  t(w, torch.float64), int(n_mu), int(n_occ), jastrow)


def run(inp: Inputs, precision: str = "bf16x3", n_orb_x: Optional[int] = None,
        events: Optional[Dict[str, list]] = None, kchunk: int = 0,
        stage_ms: Optional[list] = None, fit_mode: int = 0) -> Dict[str, object]:
    """One pass of the path.  ``events`` (name -> list) collects CUDA event
    pairs around each step; ``stage_ms`` collects the device times of the two
    W-build stages (tensor-core precisions); ``fit_mode`` 1 runs the FP64
    products of the orbitals and of the fit emulated on the tensor cores."""
    def mark(name):
        if events is None:
            return None
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        events.setdefault(name, []).append(e)
        return e

    out: Dict[str, object] = {}
    mark("a1")
    phi, dphi = api.isdf_eval_orbitals(inp.center, inp.powers, inp.exps, inp.coefs, inp.mo_coef,
                                       inp.grid, mode=fit_mode)
    mark("a1")
    mark("a2")
    piv = api.isdf_points(phi, dphi, inp.w, inp.n_mu)
    mark("a2")
    mark("a3")
    xi, xig, jit = api.isdf_fit(phi, dphi, piv, fit_mode=fit_mode)
    mark("a3")
    mark("a4")
    W, calG = api.tc_kernel_build(inp.grid, inp.w, xi, xig, inp.jastrow, precision, kchunk=kchunk,
                                  stage_ms=stage_ms if precision != "fp64" else None)
    mark("a4")
    mark("a5")
    phiP, dphiP = api.isdf_gather_pivots(phi, dphi, piv)
    nx = inp.n_occ if n_orb_x is None else n_orb_x
    D, Xp = api.xtc_density_contract(phiP, inp.n_occ, xi, inp.w, calG, nx, precision=precision)
    mark("a5")
    mark("a6")
    E = api.tc_energies(W, D, Xp, phiP, dphiP, inp.n_occ)
    mark("a6")
    out.update(phi=phi, dphi=dphi, pivots=piv, xi=xi, xig=xig, jitter=jit, W=W, calG=calG,
               D=D, Xp=Xp, phiP=phiP, dphiP=dphiP, E=E)
    return out
