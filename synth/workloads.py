"""Seeded synthetic inputs for the ISDF-xTC kernel build.

This module is input data only: geometry, integration grid, contracted
Cartesian Gaussian basis, molecular-orbital coefficients and Jastrow
parameters.  It holds none of the ISDF-xTC arithmetic (no orbital values on
the grid, no pivoting, no fitting, no kernels); both the FP64 oracle and the
CUDA path receive the arrays it produces.

Readings of what the paper leaves to PySCF (Sec. II.D, Sec. V):
  * Grid: Becke fuzzy-cell partition (Becke 1988) over atom-centred
    spheres.  Radial nodes are Gauss-Chebyshev of the second kind with the
    Becke map r = R (1 + x) / (1 - x), R = 1 bohr; angular nodes are
    equal-weight spherical Fibonacci points.  The paper uses
    Treutler-Ahlrichs radial and Lebedev angular grids (PySCF level 2); those
    tables are not reproduced here.
  * Basis: each shell is a contraction of three Cartesian primitives
    x^a y^b z^c exp(-alpha r^2) with alpha log-uniform on [0.1, 10] and
    contraction coefficients uniform on [0.5, 1.5]; every contracted function
    is normalised to unit L2 norm.
  * Orbitals: MO coefficients are standard normal and then orthonormalised in
    L2 with the analytic AO overlap (Obara-Saika), as a mean-field code would
    deliver them.  The paper's orbitals are HF or MP2 natural orbitals.
  * Jastrow: the Boys-Handy form of Eqs. bh-scaled / bh-u with the
    cusp-normalised (0,0,1) term; configs 1-2 keep only the cusp term with
    d = 1, giving u(r12) = r12 / (2 (1 + r12)).

Seeds: config k (1-based) uses seed 1000 k + 1.  Draw order from one
numpy Generator: basis exponents and contraction coefficients (atom by atom,
shell by shell), then MO coefficients, then Jastrow coefficients.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903

# Cartesian exponent tuples for angular momentum l, in a fixed order
# (a descending, then b descending).
def cart_tuples(l: int) -> List[Tuple[int, int, int]]:
    out = []
    for a in range(l, -1, -1):
        for b in range(l - a, -1, -1):
            out.append((a, b, l - a - b))
    return out


@dataclasses.dataclass
class Basis:
    """Flat list of contracted Cartesian Gaussian functions.

    Function f has centre ``center[f]`` (bohr), Cartesian powers
    ``powers[f] = (a, b, c)``, and primitives ``exps[f, k]`` with folded
    coefficients ``coefs[f, k]`` (normalisation included), k < n_prim.
    """
    center: np.ndarray   # [n_bf, 3] float64
    powers: np.ndarray   # [n_bf, 3] int32
    exps: np.ndarray     # [n_bf, n_prim] float64
    coefs: np.ndarray    # [n_bf, n_prim] float64
    atom: np.ndarray     # [n_bf] int32

    @property
    def n_bf(self) -> int:
        return int(self.center.shape[0])


@dataclasses.dataclass
class Jastrow:
    """Boys-Handy correlator parameters (Eqs. bh-scaled, bh-u).

    u2(r_i, r_j) = sum_I sum_k coef[type(I), k] *
                   [A_iI^m A_jI^n + A_jI^m A_iI^n] * E_ij^o
    with A_iI = b_I r_iI / (1 + b_I r_iI) and E_ij = d r_ij / (1 + d r_ij),
    plus, when ``cusp`` is set, the (0,0,1) term whose prefactor
    1 / (4 N_nuc d) makes the summed slope du/dr_ij at 0 equal to 1/2.
    """
    nuc_xyz: np.ndarray    # [n_nuc, 3] bohr
    nuc_type: np.ndarray   # [n_nuc] int32
    mno: np.ndarray        # [n_terms, 3] int32
    coef: np.ndarray       # [n_types, n_terms]
    b: np.ndarray          # [n_types]
    d: float
    cusp: bool = True
    # one-body nuclear-cusp term chi(r) = sum_I chi_a[t] r_I / (1 + chi_b[t] r_I),
    # entering every pair as [chi(r_i) + chi(r_j)] / (n_elec - 1); off when None
    chi_a: Optional[np.ndarray] = None   # [n_types]
    chi_b: Optional[np.ndarray] = None   # [n_types]
    n_elec: int = 0

    @property
    def n_nuc(self) -> int:
        return int(self.nuc_xyz.shape[0])

    @property
    def n_terms(self) -> int:
        return int(self.mno.shape[0])

    @property
    def n_types(self) -> int:
        return int(self.b.shape[0])

    def has_chi(self) -> bool:
        return self.chi_a is not None and bool(np.any(self.chi_a != 0.0))

    def is_radial(self) -> bool:
        """True when only the cusp term is present (u depends on r12 only)."""
        return (self.cusp and (self.n_terms == 0 or not np.any(self.coef))
                and not self.has_chi())


def with_chi(jas: Jastrow, charges, n_elec: int, beta: float = 1.0) -> Jastrow:
    """A copy of ``jas`` with the one-body cusp term: chi_a[t] = -Z_t (the
    electron-nucleus cusp slope), chi_b[t] = beta, for N = n_elec electrons."""
    a = -np.asarray(charges, dtype=np.float64).reshape(-1)
    assert a.shape[0] == jas.n_types
    return dataclasses.replace(jas, chi_a=a, chi_b=np.full(jas.n_types, float(beta)),
                               n_elec=int(n_elec))


@dataclasses.dataclass
class Workload:
    name: str
    atoms: List[str]
    xyz: np.ndarray          # [n_atom, 3] bohr
    grid_xyz: np.ndarray     # [n_g, 3]
    grid_w: np.ndarray       # [n_g]
    basis: Basis
    mo_coef: np.ndarray      # [n_bf, n_orb]
    n_occ: int
    n_mu: int
    jastrow: Jastrow
    seed: int

    @property
    def n_g(self) -> int:
        return int(self.grid_w.shape[0])

    @property
    def n_orb(self) -> int:
        return int(self.mo_coef.shape[1])


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def h_chain(n: int, spacing: float) -> Tuple[List[str], np.ndarray]:
    """Linear H_n chain along z, centred at the origin (bohr)."""
    z = (np.arange(n) - 0.5 * (n - 1)) * spacing
    xyz = np.zeros((n, 3))
    xyz[:, 2] = z
    return ["H"] * n, xyz


def h_chain_positions(z: np.ndarray) -> Tuple[List[str], np.ndarray]:
    xyz = np.zeros((len(z), 3))
    xyz[:, 2] = z - z.mean()
    return ["H"] * len(z), xyz


def benzene() -> Tuple[List[str], np.ndarray]:
    """D6h benzene in the xy plane, C-C 1.39 A, C-H 1.09 A (bohr)."""
    rc = 1.39 * BOHR_PER_ANGSTROM
    rh = rc + 1.09 * BOHR_PER_ANGSTROM
    atoms, xyz = [], []
    for k in range(6):
        t = k * math.pi / 3.0
        atoms.append("C")
        xyz.append([rc * math.cos(t), rc * math.sin(t), 0.0])
    for k in range(6):
        t = k * math.pi / 3.0
        atoms.append("H")
        xyz.append([rh * math.cos(t), rh * math.sin(t), 0.0])
    return atoms, np.array(xyz)


# --------------------------------------------------------------------------
# grid
# --------------------------------------------------------------------------

def fibonacci_sphere(n: int) -> np.ndarray:
    """n equal-area points on the unit sphere (spherical Fibonacci)."""
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def radial_chebyshev2(n: int, R: float = 1.0) -> Tuple[np.ndarray, np.ndarray]:
    """Radial nodes r_i and weights for int_0^inf F(r) r^2 dr."""
    i = np.arange(1, n + 1)
    t = i * math.pi / (n + 1)
    x = np.cos(t)
    wx = math.pi / (n + 1) * np.sin(t) ** 2
    r = R * (1.0 + x) / (1.0 - x)
    # dr/dx = 2R/(1-x)^2 ; divide by the Chebyshev weight sqrt(1 - x^2)
    w = wx * r * r * (2.0 * R / (1.0 - x) ** 2) / np.sqrt(1.0 - x * x)
    return r, w


def becke_grid(xyz: np.ndarray, n_rad: int, n_ang: int,
               R: float = 1.0) -> Tuple[np.ndarray, np.ndarray]:
    """Becke fuzzy-cell molecular grid: atom-major, then radial, then angular."""
    n_atom = xyz.shape[0]
    r, wr = radial_chebyshev2(n_rad, R)
    ang = fibonacci_sphere(n_ang)
    wa = 4.0 * math.pi / n_ang
    pts, wts = [], []
    rab = np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=2)
    for a in range(n_atom):
        p = (xyz[a][None, None, :] + r[:, None, None] * ang[None, :, :]).reshape(-1, 3)
        w0 = (wr[:, None] * wa * np.ones((1, n_ang))).reshape(-1)
        dist = np.linalg.norm(p[:, None, :] - xyz[None, :, :], axis=2)  # [np, n_atom]
        P = np.empty((p.shape[0], n_atom))
        inv_rab = 1.0 / np.where(rab > 0, rab, 1.0)
        for c0 in range(0, p.shape[0], 512):
            dd = dist[c0:c0 + 512]
            f = dd[:, :, None] - dd[:, None, :]
            f *= inv_rab[None, :, :]
            for _ in range(3):
                f3 = f * f
                f3 *= f
                f *= 1.5
                f3 *= 0.5
                f -= f3
            f *= -0.5
            f += 0.5
            idx = np.arange(n_atom)
            f[:, idx, idx] = 1.0
            P[c0:c0 + 512] = np.prod(f, axis=2)
        wb = P[:, a] / P.sum(axis=1)
        pts.append(p)
        wts.append(w0 * wb)
    grid = np.concatenate(pts, axis=0)
    w = np.concatenate(wts, axis=0)
    # positive weights (the pivot diagonal is w^2 (...)^2); Becke products
    # can underflow far inside a neighbour's cell
    w = np.maximum(w, 1e-300)
    return grid, w


# --------------------------------------------------------------------------
# basis
# --------------------------------------------------------------------------

def _overlap_1d(la: int, lb: int, a: float, b: float, A: float, B: float) -> np.ndarray:
    """Obara-Saika 1-D overlap table S[i, j], i <= la, j <= lb (vectorised over
    nothing; scalar exponents)."""
    p = a + b
    P = (a * A + b * B) / p
    S = np.zeros((la + 1, lb + 1))
    S[0, 0] = math.sqrt(math.pi / p) * math.exp(-a * b / p * (A - B) ** 2)
    for i in range(la + 1):
        for j in range(lb + 1):
            if i == 0 and j == 0:
                continue
            if i > 0:
                v = (P - A) * S[i - 1, j]
                if i > 1:
                    v += (i - 1) / (2 * p) * S[i - 2, j]
                if j > 0:
                    v += j / (2 * p) * S[i - 1, j - 1]
            else:
                v = (P - B) * S[i, j - 1]
                if j > 1:
                    v += (j - 1) / (2 * p) * S[i, j - 2]
            S[i, j] = v
    return S


def _prim_overlap(pa, a, A, pb, b, B) -> float:
    s = 1.0
    for k in range(3):
        s *= _overlap_1d(int(pa[k]), int(pb[k]), a, b, float(A[k]), float(B[k]))[pa[k], pb[k]]
    return s


def ao_overlap(basis: Basis) -> np.ndarray:
    """Analytic L2 overlap of the contracted Cartesian functions."""
    n = basis.n_bf
    S = np.zeros((n, n))
    for f in range(n):
        for h in range(f, n):
            s = 0.0
            for k in range(basis.exps.shape[1]):
                for l in range(basis.exps.shape[1]):
                    s += basis.coefs[f, k] * basis.coefs[h, l] * _prim_overlap(
                        basis.powers[f], basis.exps[f, k], basis.center[f],
                        basis.powers[h], basis.exps[h, l], basis.center[h])
            S[f, h] = S[h, f] = s
    return S


def ao_overlap_fast(basis: Basis) -> np.ndarray:
    """Vectorised analytic overlap (same result as :func:`ao_overlap`)."""
    n, npr = basis.exps.shape
    lmax = int(basis.powers.max())
    S = np.zeros((n, n))
    for k in range(npr):
        for l in range(npr):
            a = basis.exps[:, k][:, None]
            b = basis.exps[:, l][None, :]
            p = a + b
            tot = basis.coefs[:, k][:, None] * basis.coefs[:, l][None, :]
            for ax in range(3):
                A = basis.center[:, ax][:, None]
                B = basis.center[:, ax][None, :]
                P = (a * A + b * B) / p
                # OS table over (i, j) for all pairs at once
                T = {}
                T[(0, 0)] = np.sqrt(math.pi / p) * np.exp(-a * b / p * (A - B) ** 2)
                for i in range(lmax + 1):
                    for j in range(lmax + 1):
                        if i == 0 and j == 0:
                            continue
                        if i > 0:
                            v = (P - A) * T[(i - 1, j)]
                            if i > 1:
                                v = v + (i - 1) / (2 * p) * T[(i - 2, j)]
                            if j > 0:
                                v = v + j / (2 * p) * T[(i - 1, j - 1)]
                        else:
                            v = (P - B) * T[(i, j - 1)]
                            if j > 1:
                                v = v + (j - 1) / (2 * p) * T[(i, j - 2)]
                        T[(i, j)] = v
                ia = basis.powers[:, ax]
                jb = basis.powers[:, ax]
                sel = np.empty((n, n))
                for i in range(lmax + 1):
                    for j in range(lmax + 1):
                        m = (ia[:, None] == i) & (jb[None, :] == j)
                        sel = np.where(m, T[(i, j)], sel)
                tot = tot * sel
            S += tot
    return S


def make_basis(atoms: Sequence[str], xyz: np.ndarray, shells: dict,
               rng: np.random.Generator, n_prim: int = 3,
               exp_bands: Optional[dict] = None) -> Basis:
    """Draw a seeded contracted Cartesian basis.  ``shells[symbol]`` lists the
    angular momenta of the shells on that element.  Exponents are
    log-uniform on [0.1, 10]; with ``exp_bands = {l: (lo, hi)}`` the k-th of
    the n_l shells of angular momentum l draws instead from the k-th of n_l
    equal log-width bands of [lo, hi], so that many shells of one l on an atom
    stay linearly independent."""
    centers, powers, exps, coefs, atom_of = [], [], [], [], []
    for ia, sym in enumerate(atoms):
        seen = {}
        for l in shells[sym]:
            if exp_bands is None:
                lo, hi = math.log(0.1), math.log(10.0)
            else:
                k = seen.get(l, 0)
                seen[l] = k + 1
                n_l = shells[sym].count(l)
                blo, bhi = (math.log(x) for x in exp_bands[l])
                lo = blo + (bhi - blo) * k / n_l
                hi = blo + (bhi - blo) * (k + 1) / n_l
            alpha = np.exp(rng.uniform(lo, hi, size=n_prim))
            c = rng.uniform(0.5, 1.5, size=n_prim)
            for pw in cart_tuples(l):
                centers.append(xyz[ia])
                powers.append(pw)
                exps.append(alpha)
                coefs.append(c.copy())
                atom_of.append(ia)
    basis = Basis(center=np.array(centers, dtype=np.float64),
                  powers=np.array(powers, dtype=np.int32),
                  exps=np.array(exps, dtype=np.float64),
                  coefs=np.array(coefs, dtype=np.float64),
                  atom=np.array(atom_of, dtype=np.int32))
    # unit L2 norm for each contracted function
    diag = np.diag(ao_overlap_fast(basis))
    basis.coefs = basis.coefs / np.sqrt(diag)[:, None]
    return basis


def make_mo_coef(basis: Basis, n_orb: int, rng: np.random.Generator) -> np.ndarray:
    """Standard-normal MO coefficients, L2-orthonormalised with the analytic
    overlap: C <- C L^{-T} with L L^T = C^T S C."""
    S = ao_overlap_fast(basis)
    C = rng.standard_normal((basis.n_bf, n_orb))
    M = C.T @ S @ C
    L = np.linalg.cholesky(M)
    return np.linalg.solve(L, C.T).T


# --------------------------------------------------------------------------
# Jastrow
# --------------------------------------------------------------------------

# Free-term lists (reading: the paper's term list is in its absent SI).
BH_TERMS_C3 = [(0, 0, 2), (0, 0, 3), (1, 0, 0), (2, 0, 0), (3, 0, 0),
               (1, 1, 0), (2, 2, 0), (1, 1, 2), (2, 2, 2), (1, 0, 2)]


def bh_terms_c4() -> List[Tuple[int, int, int]]:
    out = []
    for m in range(4):
        for n in range(m, 4):
            for o in (0, 2, 3):
                if (m, n, o) in ((0, 0, 0), (3, 3, 3)):
                    continue
                out.append((m, n, o))
    return out


def radial_jastrow(xyz: np.ndarray, d: float = 1.0) -> Jastrow:
    """Cusp term only: u(r12) = r12 / (2 (1 + d r12))."""
    n = xyz.shape[0]
    return Jastrow(nuc_xyz=xyz.copy(), nuc_type=np.zeros(n, np.int32),
                   mno=np.zeros((0, 3), np.int32), coef=np.zeros((1, 0)),
                   b=np.ones(1), d=d, cusp=True)


def bh_jastrow(atoms: Sequence[str], xyz: np.ndarray, terms, rng,
               scale: float = 0.05, d: float = 1.0) -> Jastrow:
    types = sorted(set(atoms), key=lambda s: {"C": 0, "H": 1}.get(s, 2))
    tmap = {s: i for i, s in enumerate(types)}
    nt = np.array([tmap[s] for s in atoms], dtype=np.int32)
    coef = rng.uniform(-scale, scale, size=(len(types), len(terms)))
    return Jastrow(nuc_xyz=xyz.copy(), nuc_type=nt,
                   mno=np.array(terms, dtype=np.int32).reshape(-1, 3),
                   coef=coef, b=np.ones(len(types)), d=d, cusp=True)


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def _assemble(name, atoms, xyz, n_rad, n_ang, shells, n_orb, n_occ, n_mu,
              jkind, seed, jterms=None, jscale: float = 0.05,
              exp_bands: Optional[dict] = None) -> Workload:
    rng = np.random.default_rng(seed)
    grid, w = becke_grid(xyz, n_rad, n_ang)
    basis = make_basis(atoms, xyz, shells, rng, exp_bands=exp_bands)
    C = make_mo_coef(basis, n_orb, rng)
    if jkind == "radial":
        jas = radial_jastrow(xyz)
    else:
        jas = bh_jastrow(atoms, xyz, jterms, rng, scale=jscale)
    return Workload(name=name, atoms=list(atoms), xyz=xyz, grid_xyz=grid,
                    grid_w=w, basis=basis, mo_coef=C, n_occ=n_occ, n_mu=n_mu,
                    jastrow=jas, seed=seed)


def h6_chain() -> Workload:
    """H6 chain at 1.8 bohr, 1s1p per atom (24 orbitals), 6 x 20 x 40 grid,
    N_mu = 96, cusp-only Jastrow."""
    atoms, xyz = h_chain(6, 1.8)
    return _assemble("h6_chain", atoms, xyz, 20, 40, {"H": [0, 1]}, 24, 3, 96,
                     "radial", 1001)


def h50_chain() -> Workload:
    """H50 chain at 1.8 bohr, 2s1p1d per atom (550 functions, 400 orbitals),
    50 x 40 x 50 = 100,000 points, N_mu = 2000, cusp-only Jastrow."""
    atoms, xyz = h_chain(50, 1.8)
    return _assemble("h50_chain", atoms, xyz, 40, 50, {"H": [0, 0, 1, 2]}, 400,
                     25, 2000, "radial", 2001)


BENZENE_EXP_BANDS = {0: (0.1, 5000.0), 1: (0.1, 200.0), 2: (0.2, 40.0), 3: (0.4, 10.0)}


def benzene_c6h6() -> Workload:
    """Benzene, 100 functions per atom (12 s, 6 p, 5 d, 4 f shells), 1200
    orbitals, 12 x 75 x 302 points, N_mu = 8000, two-type BH Jastrow with 10
    terms per type.  The shells of one angular momentum take separate exponent
    bands: with all exponents in one common range the 1200-function overlap
    is numerically singular (condition ~1e15) and the orbitals cannot be
    orthonormalised; the bands bring it to ~1e9."""
    atoms, xyz = benzene()
    shells = {"C": [0] * 12 + [1] * 6 + [2] * 5 + [3] * 4,
              "H": [0] * 12 + [1] * 6 + [2] * 5 + [3] * 4}
    return _assemble("benzene", atoms, xyz, 75, 302, shells, 1200, 21, 8000,
                     "bh", 3001, BH_TERMS_C3, exp_bands=BENZENE_EXP_BANDS)


def benzene_small(n_rad: int = 6, n_ang: int = 14, n_mu: int = 64, seed: int = 3101,
                  jscale: float = 0.05, jterms=None) -> Workload:
    """Benzene geometry and two-type BH Jastrow of the benzene workload on a
    small grid (12 x n_rad x n_ang points) with an s/p basis (48 functions,
    24 orbitals, 6 occupied), for parity tests of the multi-centre kernels."""
    atoms, xyz = benzene()
    shells = {"C": [0, 1], "H": [0, 1]}
    return _assemble("benzene_small", atoms, xyz, n_rad, n_ang, shells, 24, 6, n_mu,
                     "bh", seed, BH_TERMS_C3 if jterms is None else jterms, jscale)


def h20_chain_bh() -> Workload:
    """H20 chain at 1.8 bohr, 2s2p (160 orbitals), 20 x 40 x 50 = 40,000
    points, N_mu = 800, BH Jastrow with 28 free terms (+ d, b_H)."""
    atoms, xyz = h_chain(20, 1.8)
    return _assemble("h20_chain", atoms, xyz, 40, 50, {"H": [0, 0, 1, 1]}, 160,
                     10, 800, "bh", 4001, bh_terms_c4())


def h30_chain_perturbed(k: int, n_rad: int = 40, n_ang: int = 50) -> Workload:
    """Geometry k of the perturbed H30 family: spacing s ~ U(1.6, 2.2) bohr
    plus 0.05 bohr per-atom jitter along z; 2s2p (240 orbitals), 60,000
    points, N_mu = 1200."""
    seed = 5001 + 7 * k
    rng = np.random.default_rng(seed)
    s = rng.uniform(1.6, 2.2)
    z = np.arange(30) * s + rng.uniform(-0.05, 0.05, size=30)
    atoms, xyz = h_chain_positions(z)
    return _assemble(f"h30_{k}", atoms, xyz, n_rad, n_ang, {"H": [0, 0, 1, 1]},
                     240, 15, 1200, "radial", seed + 1)


def perturbed_chain(k: int, n_atom: int = 30, n_rad: int = 40, n_ang: int = 50,
                    n_mu: int = 1200, shells=(0, 0, 1, 1), base_seed: int = 5001) -> Workload:
    """Geometry k of a perturbed H_n family: spacing s ~ U(1.6, 2.2) bohr plus
    0.05 bohr per-atom jitter along z; cusp-only Jastrow."""
    seed = base_seed + 7 * k
    rng = np.random.default_rng(seed)
    s = rng.uniform(1.6, 2.2)
    z = np.arange(n_atom) * s + rng.uniform(-0.05, 0.05, size=n_atom)
    atoms, xyz = h_chain_positions(z)
    n_orb = n_atom * sum(len(cart_tuples(l)) for l in shells)
    return _assemble(f"h{n_atom}_{k}", atoms, xyz, n_rad, n_ang, {"H": list(shells)}, n_orb,
                     n_orb // 16 or 1, n_mu, "radial", seed + 1)


def tiny_chain(n_atom: int = 2, n_rad: int = 10, n_ang: int = 16,
               shells=(0,), n_orb: Optional[int] = None, n_mu: int = 8,
               spacing: float = 1.6, seed: int = 7, jkind: str = "radial",
               jterms=None) -> Workload:
    """Small H chain for brute-force checks."""
    atoms, xyz = h_chain(n_atom, spacing)
    nbf = n_atom * sum(len(cart_tuples(l)) for l in shells)
    n_orb = nbf if n_orb is None else n_orb
    return _assemble("tiny", atoms, xyz, n_rad, n_ang, {"H": list(shells)},
                     n_orb, max(1, n_orb // 2), n_mu, jkind, seed, jterms)


CONFIGS = {
    "h6_chain": h6_chain,
    "h50_chain": h50_chain,
    "benzene": benzene_c6h6,
    "h20_chain": h20_chain_bh,
}


def seeded_matrix(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Standard-normal test matrix (e.g. an adjoint seed Wbar)."""
    return scale * np.random.default_rng(seed).standard_normal(shape)


# --------------------------------------------------------------------------
# VMC inputs (Sec. II.C): walker configurations and the sampler's random numbers
# --------------------------------------------------------------------------

def vmc_walkers(xyz: np.ndarray, n_walk: int, n_elec: int, seed: int,
                spread: float = 1.0) -> np.ndarray:
    """[n_walk][n_elec][3]: each electron on a uniformly drawn nucleus plus a
    standard-normal offset of scale `spread` bohr."""
    rng = np.random.default_rng(seed)
    at = rng.integers(0, xyz.shape[0], size=(n_walk, n_elec))
    return xyz[at] + spread * rng.standard_normal((n_walk, n_elec, 3))


def vmc_random(n_steps: int, n_elec: int, n_walk: int, seed: int):
    """Metropolis random numbers in the sampler's order: normals
    [n_steps][n_elec][n_walk][3] and uniforms [n_steps][n_elec][n_walk] in [0, 1)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n_steps, n_elec, n_walk, 3)),
            rng.random((n_steps, n_elec, n_walk)))


def vmc_chain(n_atom: int = 20, spacing: float = 1.8, seed: int = 6001,
              terms=None, jscale: float = 0.05):
    """Atoms, positions, s/p basis (4 functions per H), orthonormalised MO
    coefficients (n_occ = n_atom / 2 occupied) and BH correlator of an H chain,
    for the VMC optimisation of the correlator."""
    atoms, xyz = h_chain(n_atom, spacing)
    rng = np.random.default_rng(seed)
    basis = make_basis(atoms, xyz, {"H": [0, 1]}, rng)
    C = make_mo_coef(basis, basis.n_bf, rng)
    jas = bh_jastrow(atoms, xyz, bh_terms_c4() if terms is None else terms, rng, scale=jscale)
    return atoms, xyz, basis, C, max(1, n_atom // 2), jas
