"""Reference-variance VMC optimisation of the correlator (Sec. II.C: Eqs. Eloc,
var-loss and gn) -- oracle.

TEST INFRASTRUCTURE (FP64 numpy, plain loops over walkers and electrons).

Trial wavefunction Psi_T = F Phi_0 with F = exp(tau), tau = sum_{i<j} u(r_i, r_j)
(Eq. tau-def, u of Eqs. bh-scaled/bh-u with the cusp term and the optional
one-body term).  Phi_0 is the closed-shell reference determinant of the
n_occ occupied orbitals: electrons 0 .. n_occ-1 spin up, n_occ .. 2 n_occ-1
spin down, D_s[a][j] = phi_j(r_a) for the electrons a of spin s.

Local energy (Eq. Eloc), E_loc = (H Psi_T)/Psi_T with H the electronic
Hamiltonian plus the nuclear repulsion:
    E_loc = -1/2 sum_i [ lap_i Phi_0/Phi_0 + 2 grad_i tau . grad_i Phi_0/Phi_0
                         + lap_i tau + |grad_i tau|^2 ] + V(R),
    V = sum_{i<j} 1/r_ij - sum_{i,I} Z_I/r_iI + sum_{I<J} Z_I Z_J/R_IJ,
with grad_i Phi_0/Phi_0 = sum_j grad phi_j(r_i) (D_s^-1)[j][a(i)] and the same
with the Laplacian (the determinant's row-expansion identities).

Sampling: Metropolis moves of one electron at a time, r' = r + sigma xi
(xi standard normal), accepted when u < |Phi_0(R')/Phi_0(R)|^2; the sample is
drawn from |Phi_0|^2 and does not depend on theta (the reference-variance
protocol).  The random numbers are inputs (normals and uniforms in the order
step, electron, walker).

Objective (Eq. var-loss): raw mean m and mean absolute deviation dev of the
local energies, each clipped to [m - 5 dev, m + 5 dev], then the clipped mean
and the unbiased variance.  Update (Eq. gn): residuals r_k = E~_k - mean(E~),
C = (1/N_w) sum_k (d r_k)(d r_k)^T + lambda I, step = -eta C^-1 grad sigma^2 with
grad sigma^2 = 2/(N_w - 1) sum_k r_k d r_k.  Readings (the paper uses automatic
differentiation and does not spell these out): the clipped local energies take
the derivative of their bound, d(m +- 5 dev) with d dev = mean(sign(E_k - m)
(dE_k - dm)); d E_k / d theta by central differences of step h per parameter.
"""
from __future__ import annotations

import numpy as np

from . import jastrow as J
from . import orbitals


def ao_laplacian(basis, pts: np.ndarray) -> np.ndarray:
    """Laplacian of every contracted Cartesian Gaussian at points [n, 3] ->
    [n_bf, n]: sum over axes of d^2/dx^2 [x^p exp(-a x^2)] / exp(-a x^2) =
    p (p - 1) x^(p-2) - 2 a (2 p + 1) x^p + 4 a^2 x^(p+2), times the other two
    axes' factors."""
    n = pts.shape[0]
    nbf = basis.center.shape[0]
    lap = np.zeros((nbf, n))
    d = pts[None, :, :] - basis.center[:, None, :]
    r2 = np.sum(d * d, axis=2)
    pw = basis.powers
    for k in range(basis.exps.shape[1]):
        a = basis.exps[:, k][:, None]
        e = basis.coefs[:, k][:, None] * np.exp(-a * r2)
        vals, secs = [], []
        for ax in range(3):
            x = d[:, :, ax]
            p = pw[:, ax][:, None]
            vals.append(x ** p)
            second = (np.where(p > 1, p * (p - 1) * x ** np.maximum(p - 2, 0), 0.0)
                      - 2.0 * a * (2 * p + 1) * x ** p + 4.0 * a * a * x ** (p + 2))
            secs.append(second)
        for ax in range(3):
            term = secs[ax]
            for bx in range(3):
                if bx != ax:
                    term = term * vals[bx]
            lap += term * e
    return lap


def occupied_orbitals(basis, c_occ: np.ndarray, R: np.ndarray):
    """phi [n_occ][N], grad [3][n_occ][N], Laplacian [n_occ][N] of the occupied
    orbitals (columns of c_occ) at the electron positions R [N, 3]."""
    v, g = orbitals.eval_ao(basis, R)
    lap = ao_laplacian(basis, R)
    CT = c_occ.T
    return CT @ v, np.stack([CT @ g[c] for c in range(3)]), CT @ lap


def lap1_u(ri: np.ndarray, rj: np.ndarray, jas) -> np.ndarray:
    """Laplacian of u(r_i, r_j) with respect to r_i for all pairs [n, m]
    (analytic; the self pair is not excluded here).  With A(r) = b r/(1 + b r)
    and E(r) = d r/(1 + d r): A' = b/(1+br)^2, A'' = -2 b^2/(1+br)^3, lap A =
    A'' + 2 A'/r (likewise E), and for a term S(A_i) E^o (S = A_i^m A_j^n + A_j^m A_i^n)
      lap = S'' E^o |grad A_i|^2 + S' E^o lap A_i + 2 S' o E^(o-1) grad A_i . grad E
            + S [o (o-1) E^(o-2) |grad E|^2 + o E^(o-1) lap E]."""
    dv = ri[:, None, :] - rj[None, :, :]
    r = np.sqrt(np.sum(dv * dv, axis=2))
    with np.errstate(invalid="ignore", divide="ignore"):
        eij = np.where(r[..., None] > 0, dv / r[..., None], 0.0)
        rinv = np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), 0.0)
    d = jas.d
    den = 1.0 + d * r
    E = d * r / den
    E1 = d / den ** 2
    E2 = -2.0 * d * d / den ** 3
    lapE = E2 + 2.0 * E1 * rinv
    out = np.zeros_like(r)
    if jas.cusp:
        out += lapE / (2.0 * d)
    for I in range(jas.n_nuc):
        t = jas.nuc_type[I]
        b = jas.b[t]
        dvi = ri - jas.nuc_xyz[I]
        riI = np.linalg.norm(dvi, axis=1)
        rjI = np.linalg.norm(rj - jas.nuc_xyz[I], axis=1)
        with np.errstate(invalid="ignore", divide="ignore"):
            eI = np.where(riI[:, None] > 0, dvi / riI[:, None], 0.0)
            rIinv = np.where(riI > 0, 1.0 / np.where(riI > 0, riI, 1.0), 0.0)
        dni = 1.0 + b * riI
        Ai = (b * riI / dni)[:, None]
        A1 = (b / dni ** 2)[:, None]
        A2 = (-2.0 * b * b / dni ** 3)[:, None]
        lapA = A2 + 2.0 * A1 * rIinv[:, None]
        Aj = (b * rjI / (1.0 + b * rjI))[None, :]
        cos = np.einsum("nc,nmc->nm", eI, eij)          # e_iI . e_ij
        for k in range(jas.n_terms):
            m, n, o = (int(x) for x in jas.mno[k])
            c = jas.coef[t, k]
            S = Ai ** m * Aj ** n + Aj ** m * Ai ** n
            S1 = (m * Ai ** max(m - 1, 0) * Aj ** n if m > 0 else 0.0) + \
                 (n * Aj ** m * Ai ** max(n - 1, 0) if n > 0 else 0.0)
            S2 = (m * (m - 1) * Ai ** max(m - 2, 0) * Aj ** n if m > 1 else 0.0) + \
                 (n * (n - 1) * Aj ** m * Ai ** max(n - 2, 0) if n > 1 else 0.0)
            Eo = E ** o
            Eo1 = o * E ** (o - 1) if o > 0 else 0.0
            Eo2 = o * (o - 1) * E ** (o - 2) if o > 1 else 0.0
            out += c * (S2 * Eo * A1 ** 2 + S1 * Eo * lapA + 2.0 * S1 * Eo1 * A1 * E1 * cos
                        + S * (Eo2 * E1 ** 2 + Eo1 * lapE))
    if J.chi_on(jas):
        lchi = np.zeros(ri.shape[0])
        for I in range(jas.n_nuc):
            t = jas.nuc_type[I]
            rI = np.linalg.norm(ri - jas.nuc_xyz[I], axis=1)
            den_c = 1.0 + jas.chi_b[t] * rI
            c1 = jas.chi_a[t] / den_c ** 2
            c2 = -2.0 * jas.chi_a[t] * jas.chi_b[t] / den_c ** 3
            with np.errstate(invalid="ignore", divide="ignore"):
                lchi += c2 + np.where(rI > 0, 2.0 * c1 / np.where(rI > 0, rI, 1.0), 0.0)
        out += lchi[:, None] / (jas.n_elec - 1)
    return out


def local_energy(R: np.ndarray, basis, c_occ: np.ndarray, jas, nuc_xyz: np.ndarray,
                 charges: np.ndarray) -> float:
    """E_loc of one configuration R [N, 3] (N = 2 n_occ), Eq. Eloc."""
    n_occ = c_occ.shape[1]
    N = 2 * n_occ
    phi, dphi, lphi = occupied_orbitals(basis, c_occ, R)
    gphi = np.zeros((N, 3))
    lphi0 = np.zeros(N)
    for s in range(2):
        idx = np.arange(s * n_occ, (s + 1) * n_occ)
        D = phi[:, idx].T                                # [a][j] = phi_j(r_a)
        Dinv = np.linalg.inv(D)                          # [j][a]
        for a_loc, a in enumerate(idx):
            col = Dinv[:, a_loc]
            gphi[a] = np.array([dphi[c][:, a] @ col for c in range(3)])
            lphi0[a] = lphi[:, a] @ col
    g = J.grad1_u(R, R, jas)                             # [3, N, N]
    lu = lap1_u(R, R, jas)                               # [N, N]
    off = ~np.eye(N, dtype=bool)
    gtau = np.stack([np.sum(np.where(off, g[c], 0.0), axis=1) for c in range(3)], axis=1)
    ltau = np.sum(np.where(off, lu, 0.0), axis=1)
    kin = -0.5 * np.sum(lphi0 + 2.0 * np.sum(gtau * gphi, axis=1) + ltau
                        + np.sum(gtau * gtau, axis=1))
    V = 0.0
    for i in range(N):
        for j in range(i + 1, N):
            V += 1.0 / np.linalg.norm(R[i] - R[j])
        for I in range(nuc_xyz.shape[0]):
            V -= charges[I] / np.linalg.norm(R[i] - nuc_xyz[I])
    for I in range(nuc_xyz.shape[0]):
        for K in range(I + 1, nuc_xyz.shape[0]):
            V += charges[I] * charges[K] / np.linalg.norm(nuc_xyz[I] - nuc_xyz[K])
    return float(kin + V)


def local_energies(walkers: np.ndarray, basis, c_occ, jas, nuc_xyz, charges) -> np.ndarray:
    """E_loc for every walker [N_w][N][3]."""
    return np.array([local_energy(w, basis, c_occ, jas, nuc_xyz, charges) for w in walkers])


def metropolis(walkers: np.ndarray, basis, c_occ: np.ndarray, normals: np.ndarray,
               uniforms: np.ndarray, sigma: float):
    """Single-electron Metropolis sweeps on |Phi_0|^2.  normals [S][N][N_w][3],
    uniforms [S][N][N_w]; returns the moved walkers and the accepted count.
    The ratio is the determinant quotient, recomputed from both determinants."""
    W = walkers.copy()
    n_occ = c_occ.shape[1]
    acc = 0
    S, N, Nw = uniforms.shape
    for s in range(S):
        for i in range(N):
            spin = i // n_occ
            idx = np.arange(spin * n_occ, (spin + 1) * n_occ)
            for w in range(Nw):
                R = W[w]
                phi_old, _, _ = occupied_orbitals(basis, c_occ, R[idx])
                Rn = R[idx].copy()
                Rn[i - spin * n_occ] = R[i] + sigma * normals[s, i, w]
                phi_new, _, _ = occupied_orbitals(basis, c_occ, Rn)
                q = np.linalg.det(phi_new.T) / np.linalg.det(phi_old.T)
                if uniforms[s, i, w] < q * q:
                    W[w, i] = Rn[i - spin * n_occ]
                    acc += 1
    return W, acc


def clipped_objective(E: np.ndarray):
    """Eq. var-loss: clipped energies, their mean and unbiased variance."""
    m = float(np.mean(E))
    dev = float(np.mean(np.abs(E - m)))
    Ec = np.clip(E, m - 5.0 * dev, m + 5.0 * dev)
    mean = float(np.mean(Ec))
    var = float(np.sum((Ec - mean) ** 2) / (len(E) - 1))
    return Ec, mean, var


def residual_jacobian(E: np.ndarray, dE: np.ndarray) -> np.ndarray:
    """d r_k / d theta [P][N_w] for r_k = E~_k - mean(E~), from d E_k [P][N_w],
    with clipped energies following their bound (module docstring)."""
    m = np.mean(E)
    dev = np.mean(np.abs(E - m))
    dm = np.mean(dE, axis=1)
    sgn = np.sign(E - m)
    ddev = np.mean(sgn[None, :] * (dE - dm[:, None]), axis=1)
    lo, hi = m - 5.0 * dev, m + 5.0 * dev
    dEc = dE.copy()
    low, high = E < lo, E > hi
    dEc[:, low] = (dm - 5.0 * ddev)[:, None]
    dEc[:, high] = (dm + 5.0 * ddev)[:, None]
    return dEc - np.mean(dEc, axis=1)[:, None]


def gauss_newton_step(E: np.ndarray, dE: np.ndarray, lam: float, eta: float) -> np.ndarray:
    """Eq. gn: C = (1/N_w) sum_k dr_k dr_k^T + lam I, step = -eta C^-1 grad sigma^2."""
    Ec, mean, _ = clipped_objective(E)
    r = Ec - mean
    dr = residual_jacobian(E, dE)
    Nw = len(E)
    C = dr @ dr.T / Nw + lam * np.eye(dr.shape[0])
    grad = 2.0 / (Nw - 1) * dr @ r
    return -eta * np.linalg.solve(C, grad)


def energy_jacobian_fd(walkers, basis, c_occ, jas, nuc_xyz, charges, h: float = 1e-5):
    """d E_loc / d theta [P][N_w] by central differences of step h, theta =
    (d, b_0 .. b_{T-1}, c row-major) as in the adjoint oracle."""
    from . import adjoint
    th = adjoint.get_theta(jas)
    out = np.zeros((len(th), walkers.shape[0]))
    for p in range(len(th)):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        Ep = local_energies(walkers, basis, c_occ, adjoint.set_theta(jas, tp), nuc_xyz, charges)
        Em = local_energies(walkers, basis, c_occ, adjoint.set_theta(jas, tm), nuc_xyz, charges)
        out[p] = (Ep - Em) / (2 * h)
    return out
