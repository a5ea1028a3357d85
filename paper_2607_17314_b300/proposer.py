"""Learned interpolation-point proposer (the paper has no learned
component).  Python driver of the libisdftc kernels: feature
extraction, training by weighted binary cross-entropy against the plain
pivoted-Cholesky selection, and proposal = pivoted Cholesky restricted to the
kappa N_mu highest-scoring points, scored by the scalar-channel fit error
against the plain selection (the fallback)."""
from __future__ import annotations

import ctypes
import dataclasses
from typing import List, Optional

import numpy as np
import torch

from . import _capi as C
from .api import _dims, _orbital_planes, _ptr, _reqs, _shape, _stream, _ws

f32, f64 = torch.float32, torch.float64


def n_params() -> int:
    """Number of FP32 parameters of the 8 -> 128 -> 128 -> 1 network."""
    return int(C.load().isdf_mlp_n_params())


def features(phi, dphi, w, grid_xyz, nuc_xyz) -> torch.Tensor:
    """Per-point features [n_g][8] (pivot diagonals of Alg. 1 and its gradient
    branch, weights, densities, nucleus distances) on the device."""
    lib = C.load()
    n_orb, n_g = _orbital_planes(phi, dphi, lambda n_g: (w, f64, "w", (n_g,)),
                                 lambda n_g: (grid_xyz, f64, "grid_xyz", (n_g, 3)))
    nuc = np.ascontiguousarray(np.asarray(nuc_xyz, dtype=np.float64).reshape(-1, 3))
    feat = torch.empty((n_g, 8), dtype=f32, device=phi.device)
    C.check("isdf_mlp_features", lib.isdf_mlp_features(
        _ptr(phi), _ptr(dphi), _ptr(w), _ptr(grid_xyz), n_g, n_orb,
        nuc.ctypes.data_as(ctypes.c_void_p), nuc.shape[0], _ptr(feat), _stream()))
    return feat


def forward(params, feat) -> torch.Tensor:
    """Scores [n] of the network with BF16-rounded weights."""
    lib = C.load()
    _shape(feat, "feat", (None, 8))
    _reqs((params, f32, "params", (n_params(),)), (feat, f32, "feat", None))
    scores = torch.empty(feat.shape[0], dtype=f32, device=feat.device)
    C.check("isdf_mlp_forward", lib.isdf_mlp_forward(_ptr(params), _ptr(feat), feat.shape[0],
                                                     _ptr(scores), _stream()))
    return scores


def backward(params, feat, labels, pos_w: float, n_total: int, grad, loss):
    """Add the weighted-BCE gradient (normalised by n_total) to grad and the
    unnormalised loss sum to loss (device FP64 [1])."""
    lib = C.load()
    n, P = _shape(feat, "feat", (None, 8))[0], n_params()
    _reqs((params, f32, "params", (P,)), (feat, f32, "feat", None), (labels, f32, "labels", (n,)),
          (grad, f32, "grad", (P,)), (loss, f64, "loss", (1,)))
    C.check("isdf_mlp_backward", lib.isdf_mlp_backward(
        _ptr(params), _ptr(feat), _ptr(labels), feat.shape[0], float(pos_w), int(n_total),
        _ptr(grad), _ptr(loss), _stream()))


def adam(params, grad, m, v, step: int, lr: float):
    """One bias-corrected Adam step on params (1-based step)."""
    lib = C.load()
    P = n_params()
    _reqs(*[(t, f32, name, (P,)) for t, name in ((params, "params"), (grad, "grad"), (m, "m"),
                                                 (v, "v"))])
    C.check("isdf_mlp_adam", lib.isdf_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v),
                                               int(step), float(lr), _stream()))


def topk(scores, k: int) -> torch.Tensor:
    """Indices of the k highest scores, ties by the lower index, ascending."""
    lib = C.load()
    _reqs((scores, f32, "scores", (None,)))
    out = torch.empty(k, dtype=torch.int32, device=scores.device)
    C.check("isdf_mlp_topk", lib.isdf_mlp_topk(_ptr(scores), scores.shape[0], int(k), _ptr(out),
                                               _stream()))
    return out


def points_restricted(phi, dphi, w, cand, n_mu: int) -> torch.Tensor:
    """Fused pivoted Cholesky (Alg. 1 and Sec. II.D) on the candidate points
    only; grid indices of the selected points (fewer if the rank runs out)."""
    lib = C.load()
    n_orb, n_g = _orbital_planes(phi, dphi, lambda n_g: (w, f64, "w", (n_g,)),
                                 lambda _: (cand, torch.int32, "cand", (None,)))
    piv = torch.empty(n_mu, dtype=torch.int32, device=phi.device)
    n_out = C.INT(0)
    ws = _ws(lib.isdf_points_restricted_workspace(cand.numel(), n_orb, n_mu), phi.device)
    st = lib.isdf_points_restricted(_ptr(phi), _ptr(dphi), _ptr(w), n_g, n_orb, _ptr(cand),
                                    cand.numel(), n_mu, _ptr(piv), ctypes.byref(n_out), _ptr(ws),
                                    ws.numel(), _stream())
    C.check("isdf_points_restricted", st, allow=(C.ISDF_E_RANK,))
    return piv[:n_out.value]


def fit_error(phi, w, pivots) -> float:
    """Scalar-channel weighted ISDF fit error of a pivot set (Eq. isdf-rho)."""
    lib = C.load()
    n_orb, n_g = _dims(phi, "phi", 2)
    _reqs((phi, f64, "phi", None), (w, f64, "w", (n_g,)), (pivots, torch.int32, "pivots", (None,)))
    eps = ctypes.c_double(0.0)
    ws = _ws(lib.isdf_fit_error_workspace(n_g, n_orb, pivots.numel()), phi.device)
    C.check("isdf_fit_error", lib.isdf_fit_error(_ptr(phi), _ptr(w), n_g, n_orb, _ptr(pivots),
                                                 pivots.numel(), ctypes.byref(eps), _ptr(ws),
                                                 ws.numel(), _stream()))
    return float(eps.value)


def init_params(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-initialised FP32 parameters (layout of include/isdftc.h)."""
    rng = np.random.default_rng(seed)
    H, F = 128, 8
    W1 = rng.standard_normal((H, F)) * np.sqrt(2.0 / F)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
    W3 = rng.standard_normal(H) * np.sqrt(1.0 / H)
    th = np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3, [0.0]])
    return torch.tensor(th, dtype=f32, device=device)


@dataclasses.dataclass
class Sample:
    """One training geometry: features, labels (plain selection) and the
    arrays needed to score a proposal."""
    feat: torch.Tensor
    labels: torch.Tensor
    phi: torch.Tensor
    dphi: torch.Tensor
    w: torch.Tensor
    plain: torch.Tensor
    n_mu: int


class Proposer:
    """The network, its Adam state, training on plain selections and proposals
    with the plain selection as fallback."""

    def __init__(self, seed: int = 0, lr: float = 1e-3, device="cuda"):
        self.params = init_params(seed, device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=f64, device=device)
        self.step = 0
        self.lr = lr

    def train_epoch(self, samples: List[Sample]) -> float:
        """One Adam step per geometry; returns the mean loss over the epoch."""
        tot, npts = 0.0, 0
        for smp in samples:
            n = smp.feat.shape[0]
            pos_w = float((n - smp.n_mu) / max(smp.n_mu, 1))
            self.grad.zero_()
            self.loss.zero_()
            backward(self.params, smp.feat, smp.labels, pos_w, n, self.grad, self.loss)
            self.step += 1
            adam(self.params, self.grad, self.m, self.v, self.step, self.lr)
            tot += float(self.loss.item())
            npts += n
        return tot / npts

    def propose(self, smp: Sample, kappa: float = 3.0) -> torch.Tensor:
        """Pivots from the kappa N_mu highest-scoring candidates."""
        scores = forward(self.params, smp.feat)
        k = min(int(kappa * smp.n_mu), smp.feat.shape[0])
        cand = topk(scores, k)
        return points_restricted(smp.phi, smp.dphi, smp.w, cand, smp.n_mu)

    def candidates(self, smp: Sample, kappa: float = 3.0) -> torch.Tensor:
        """The kappa N_mu highest-scoring points of the network."""
        scores = forward(self.params, smp.feat)
        return topk(scores, min(int(kappa * smp.n_mu), smp.feat.shape[0]))

    def select(self, smp: Sample, kappa: float = 3.0, tolerance: float = 2.0):
        """Proposal if its fit error is within `tolerance` x the plain
        selection's, else the plain selection (fallback)."""
        piv = self.propose(smp, kappa)
        e_prop = fit_error(smp.phi, smp.w, piv) if piv.numel() == smp.n_mu else float("inf")
        e_plain = fit_error(smp.phi, smp.w, smp.plain)
        if e_prop <= tolerance * e_plain:
            return piv, e_prop, e_plain, False
        return smp.plain, e_prop, e_plain, True


def diagonal_candidates(smp: Sample, kappa: float = 3.0) -> torch.Tensor:
    """The same candidate budget without the network: the kappa N_mu points with
    the largest initial scalar pivot diagonal w^2 rho^2 (the quantity the
    first step of Alg. 1 maximises; feature 0)."""
    d0 = smp.feat[:, 0].contiguous()
    return topk(d0, min(int(kappa * smp.n_mu), smp.feat.shape[0]))


def recall(cand: torch.Tensor, plain: torch.Tensor) -> float:
    """Fraction of the plain selection's points inside a candidate set."""
    return float(torch.isin(plain.long(), cand.long()).float().mean())
