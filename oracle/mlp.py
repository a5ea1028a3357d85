"""Learned interpolation-point proposer -- oracle (not in the paper, which
selects points by pivoted Cholesky only).

TEST INFRASTRUCTURE (FP64 numpy on the same BF16-rounded weights the GPU uses).

Features per grid point (F = 8), from the quantities Alg. 1 works with:
  f0 = log10(w^2 rho^2 + 1e-300) / 10      scalar pivot diagonal D^(phi)
  f1 = log10(w^2 rho tau + 1e-300) / 10    gradient pivot diagonal D^(grad)
  f2 = log10(w + 1e-300) / 10
  f3 = log10(rho + 1e-300) / 10            rho = sum_p phi_p^2
  f4 = log10(tau + 1e-300) / 10            tau = sum_{p,c} (d_c phi_p)^2
  f5 = r_1 / 5,  f6 = r_2 / 5              distances to the two nearest nuclei (bohr)
  f7 = log10(r_1 + 1e-3)
Model: s = W3 relu(W2 relu(W1 x + b1) + b2) + b3 (widths 8 -> 128 -> 128 -> 1).
Loss: weighted binary cross-entropy with logits against y = 1 for the points the
plain pivoted Cholesky selects, positive weight pos_w:
  l = pos_w y softplus(-s) + (1 - y) softplus(s), averaged over points.
Optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8) on FP32 master weights; the
forward uses their BF16 roundings.
Selection: the kappa * N_mu highest-scoring points form the candidate set; the
plain pivoted Cholesky (Alg. 1 + fusion) runs on that set only.
Fit error: eps = sum_g w_g^2 r_g / sum_g w_g^2 D0_g with r_g the scalar-channel
ISDF residual of the full grid (the weighted Frobenius residual of Eq. isdf-rho).
"""
from __future__ import annotations

import numpy as np

F = 8
H = 128
N_PARAMS = H * F + H + H * H + H + H + 1


def features(phi, dphi, w, grid, nuc_xyz):
    """Per-point features [n_g][8]: log10 of the scalar and gradient pivot
    diagonals (Alg. 1 and its gradient branch, Sec. II.D), of w, rho and tau
    (each / 10), the two nearest-nucleus distances / 5 and log10(r_1 + 1e-3)."""
    rho = np.sum(phi * phi, axis=0)
    tau = np.sum(dphi * dphi, axis=(0, 1))
    dist = np.linalg.norm(grid[:, None, :] - nuc_xyz[None, :, :], axis=2)
    ds = np.sort(dist, axis=1)
    r1 = ds[:, 0]
    r2 = ds[:, 1] if ds.shape[1] > 1 else ds[:, 0]
    f = np.stack([
        np.log10(w * w * rho * rho + 1e-300) / 10.0,
        np.log10(w * w * rho * tau + 1e-300) / 10.0,
        np.log10(w + 1e-300) / 10.0,
        np.log10(rho + 1e-300) / 10.0,
        np.log10(tau + 1e-300) / 10.0,
        r1 / 5.0,
        r2 / 5.0,
        np.log10(r1 + 1e-3),
    ], axis=1)
    return f


def unpack(theta):
    """theta (flat, FP64) -> W1 [H][F], b1 [H], W2 [H][H], b2 [H], W3 [H], b3 []."""
    o = 0
    W1 = theta[o:o + H * F].reshape(H, F); o += H * F
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    W3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, W3, b3


def bf16_round(x):
    """Round FP64 values to the nearest BF16 (through FP32, ties to even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed: int = 0) -> np.ndarray:
    """He-scaled normal initial weights and zero biases, flattened (unpack order)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((H, F)) * np.sqrt(2.0 / F)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
    W3 = rng.standard_normal(H) * np.sqrt(1.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3, [0.0]])


def forward(theta, x, rounding: bool = True):
    """Scores and activations with BF16-rounded weights (biases included);
    rounding=False evaluates the same network on the unrounded weights."""
    W1, b1, W2, b2, W3, b3 = unpack(bf16_round(theta) if rounding else theta)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    s = h2 @ W3 + b3
    return s, (x, z1, h1, z2, h2)


def softplus(t):
    """log(1 + e^t) without overflow."""
    return np.maximum(t, 0.0) + np.log1p(np.exp(-np.abs(t)))


def loss_and_grad(theta, x, y, pos_w, rounding: bool = True):
    """Mean weighted BCE and its gradient with respect to theta (through the
    BF16-rounded weights, i.e. the straight-through gradient)."""
    W1, b1, W2, b2, W3, b3 = unpack(bf16_round(theta) if rounding else theta)
    s, (x, z1, h1, z2, h2) = forward(theta, x, rounding)
    n = x.shape[0]
    l = np.mean(pos_w * y * softplus(-s) + (1.0 - y) * softplus(s))
    sig = 1.0 / (1.0 + np.exp(-s))
    ds = (pos_w * y * (sig - 1.0) + (1.0 - y) * sig) / n
    gW3 = h2.T @ ds
    gb3 = np.sum(ds)
    d2 = np.outer(ds, W3) * (z2 > 0)
    gW2 = d2.T @ h1
    gb2 = np.sum(d2, axis=0)
    d1 = (d2 @ W2) * (z1 > 0)
    gW1 = d1.T @ x
    gb1 = np.sum(d1, axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return float(l), g


def adam(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step (Kingma and Ba) at 1-based step t."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def candidates(scores, k):
    """Indices of the k highest scores (ascending index order; ties by index)."""
    order = np.lexsort((np.arange(scores.shape[0]), -scores))
    return np.sort(order[:k])


def fit_error(phi, w, piv):
    """eps = sum w^2 r / sum w^2 D0 for the scalar channel (Eq. isdf-rho)."""
    from . import fit
    xi, _, _ = fit.fit(phi, np.zeros((3,) + phi.shape), piv, channels=(0,))
    r = fit.fit_residual(phi, w, piv, xi)
    rho = np.sum(phi * phi, axis=0)
    return float(np.sum(r) / np.sum(w * w * rho * rho))
