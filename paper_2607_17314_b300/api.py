"""Python front end of libisdftc with the C ABI's names.

Each function takes CUDA tensors, allocates the outputs and the workspace
with torch (device memory only), and calls the matching C entry point on the
current torch stream.  There is no host or fallback implementation: on a
machine without the built library or without a GPU these functions raise.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

import torch

from . import _capi as C

f64 = torch.float64


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ws(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _req(t: torch.Tensor, dtype, name: str):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t


def _shape(t: torch.Tensor, name: str, shape) -> tuple:
    """t's shape after checking it against `shape` (None entries match any
    size).  The library reads and writes exactly the sizes it is passed, so a
    tensor smaller than they say would be accessed out of bounds on the device."""
    if t.dim() != len(shape) or any(want is not None and got != want
                                    for got, want in zip(t.shape, shape)):
        want = tuple("*" if x is None else x for x in shape)
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {want}")
    return tuple(t.shape)


def _dims(t: torch.Tensor, name: str, rank: int) -> tuple:
    return _shape(t, name, (None,) * rank)


def _reqs(*specs):
    """specs: (tensor, dtype, name, shape or None).  Every shape is checked
    before any dtype, layout or device, so the host-side size checks run (and
    are testable) without a GPU; then every tensor must be a contiguous CUDA
    tensor of its dtype."""
    for t, _, name, shape in specs:
        if shape is not None:
            _shape(t, name, shape)
    for t, dtype, name, _ in specs:
        _req(t, dtype, name)


def _orbital_planes(phi, dphi, *more):
    """(n_orb, n_g) of phi [n_orb][n_g]; phi, dphi [3][n_orb][n_g] and the
    further specs (built from n_g by the caller's lambda) checked."""
    n_orb, n_g = _dims(phi, "phi", 2)
    _reqs((phi, f64, "phi", None), (dphi, f64, "dphi", (3, n_orb, n_g)),
          *[m(n_g) for m in more])
    return n_orb, n_g


def _factors(W, D, Xp, phi_piv, dphi_piv, x_rows_min=None):
    """(n_mu, n_orb) of the pivot factors, with W [4][n_mu][n_mu], D [n_mu][n_mu],
    dphi_piv [3][n_mu][n_orb] and the packed X [rows][n_mu] checked: at least
    x_rows_min rows when given, else the full X of all n_orb orbitals."""
    n_mu, n_orb = _dims(phi_piv, "phi_piv", 2)
    _shape(Xp, "Xp", (None, n_mu))
    full = n_orb * (n_orb + 1) // 2
    if x_rows_min is not None and Xp.shape[0] < x_rows_min:
        raise ValueError(f"Xp has {Xp.shape[0]} rows, needs at least {x_rows_min}")
    if x_rows_min is None and Xp.shape[0] != full:
        raise ValueError(f"Xp has {Xp.shape[0]} rows; the full X of {n_orb} orbitals has {full}")
    _reqs((phi_piv, f64, "phi_piv", None), (dphi_piv, f64, "dphi_piv", (3, n_mu, n_orb)),
          (W, f64, "W", (4, n_mu, n_mu)), (D, f64, "D", (n_mu, n_mu)), (Xp, f64, "Xp", None))
    return n_mu, n_orb


def jastrow_struct(nuc_xyz, nuc_type, mno, coef, b, d: float, cusp: bool = True,
                   chi_a=None, chi_b=None, n_elec: int = 0) -> C.IsdfJastrow:
    """Fill the host isdf_jastrow struct from arrays (see include/isdftc.h);
    chi_a/chi_b (per type) and n_elec give the one-body term of Eq. tau-def."""
    import numpy as np
    J = C.IsdfJastrow()
    nuc_xyz = np.asarray(nuc_xyz, dtype=np.float64).reshape(-1, 3)
    mno = np.asarray(mno, dtype=np.int32).reshape(-1, 3)
    coef = np.asarray(coef, dtype=np.float64).reshape(len(np.atleast_1d(b)), -1)
    b = np.atleast_1d(np.asarray(b, dtype=np.float64))
    if nuc_xyz.shape[0] > C.ISDF_MAX_NUC or mno.shape[0] > C.ISDF_MAX_TERMS or b.shape[0] > C.ISDF_MAX_TYPES:
        raise ValueError("Jastrow exceeds the library limits")
    J.n_nuc, J.n_types, J.n_terms, J.cusp, J.d = nuc_xyz.shape[0], b.shape[0], mno.shape[0], int(cusp), float(d)
    for I in range(nuc_xyz.shape[0]):
        for c in range(3):
            J.nuc_xyz[I][c] = float(nuc_xyz[I, c])
        J.nuc_type[I] = int(nuc_type[I])
    for t in range(b.shape[0]):
        J.b[t] = float(b[t])
        for k in range(mno.shape[0]):
            J.coef[t][k] = float(coef[t, k])
    for k in range(mno.shape[0]):
        for c in range(3):
            J.mno[k][c] = int(mno[k, c])
    if chi_a is not None:
        ca = np.atleast_1d(np.asarray(chi_a, dtype=np.float64))
        cb = np.atleast_1d(np.asarray(chi_b, dtype=np.float64))
        if ca.shape[0] != b.shape[0] or cb.shape[0] != b.shape[0]:
            raise ValueError("chi_a and chi_b need one value per nucleus type")
        for t in range(b.shape[0]):
            J.chi_a[t] = float(ca[t])
            J.chi_b[t] = float(cb[t])
        J.n_elec = int(n_elec)
    return J


def jastrow_from(obj) -> C.IsdfJastrow:
    """isdf_jastrow from any object with nuc_xyz, nuc_type, mno, coef, b, d, cusp
    (and optionally chi_a, chi_b, n_elec)."""
    return jastrow_struct(obj.nuc_xyz, obj.nuc_type, obj.mno, obj.coef, obj.b, obj.d, obj.cusp,
                          getattr(obj, "chi_a", None), getattr(obj, "chi_b", None),
                          getattr(obj, "n_elec", 0))


def isdf_eval_orbitals(center, powers, exps, coefs, mo_coef, grid_xyz,
                       mode: int = 0) -> Tuple[torch.Tensor, torch.Tensor]:
    """phi [n_orb][n_g], dphi [3][n_orb][n_g] (Alg. 2 step 2); mode 1 takes
    the contractions as FP64 products emulated on the tensor cores."""
    lib = C.load()
    dev = grid_xyz.device
    n_bf = _dims(exps, "exps", 2)[0]
    n_orb = _shape(mo_coef, "mo_coef", (n_bf, None))[1]
    n_g = _shape(grid_xyz, "grid_xyz", (None, 3))[0]
    basis = _basis(center, powers, exps, coefs, (mo_coef, f64, "mo_coef", None),
                   (grid_xyz, f64, "grid_xyz", None))
    phi = torch.empty((n_orb, n_g), dtype=f64, device=dev)
    dphi = torch.empty((3, n_orb, n_g), dtype=f64, device=dev)
    if mode == 0:
        ws = _ws(lib.isdf_eval_orbitals_workspace(n_bf, n_g), dev)
        C.check("isdf_eval_orbitals", lib.isdf_eval_orbitals(
            ctypes.byref(basis), _ptr(mo_coef), n_orb, _ptr(grid_xyz), n_g, _ptr(phi),
            _ptr(dphi), _ptr(ws), ws.numel(), _stream()))
    else:
        ws = _ws(lib.isdf_eval_orbitals_workspace_mode(n_bf, n_g, n_orb, int(mode)), dev)
        C.check("isdf_eval_orbitals_mode", lib.isdf_eval_orbitals_mode(
            ctypes.byref(basis), _ptr(mo_coef), n_orb, _ptr(grid_xyz), n_g, _ptr(phi),
            _ptr(dphi), int(mode), _ptr(ws), ws.numel(), _stream()))
    return phi, dphi


def isdf_points(phi, dphi, w, n_mu: int, mode: int = 0, allow_rank: bool = False):
    """Interpolation points (Alg. 1 + fusion): int32 tensor of length n_mu_out."""
    lib = C.load()
    dev = phi.device
    n_orb, n_g = _orbital_planes(phi, dphi, lambda n_g: (w, f64, "w", (n_g,)))
    piv = torch.empty(n_mu, dtype=torch.int32, device=dev)
    out = C.INT(0)
    ws = _ws(lib.isdf_points_workspace(n_g, n_mu), dev)
    st = lib.isdf_points(_ptr(phi), _ptr(dphi), _ptr(w), n_g, n_orb, n_mu, mode, _ptr(piv),
                         ctypes.byref(out), _ptr(ws), ws.numel(), _stream())
    C.check("isdf_points", st, allow=(C.ISDF_E_RANK,) if allow_rank else ())
    return piv[:out.value]


def isdf_points_fixed_rank(phi, dphi, w, n_ch_phi: int, n_ch_grad: int,
                           allow_rank: bool = False):
    """The paper's pivot fusion (Sec. II.D): each channel to its own rank, then
    the union (scalar pivots first).  int32 tensor of length n_mu_out."""
    lib = C.load()
    dev = phi.device
    n_orb, n_g = _orbital_planes(phi, dphi, lambda n_g: (w, f64, "w", (n_g,)))
    piv = torch.empty(max(n_ch_phi + n_ch_grad, 1), dtype=torch.int32, device=dev)
    out = C.INT(0)
    ws = _ws(lib.isdf_points_fixed_rank_workspace(n_g, n_ch_phi, n_ch_grad), dev)
    st = lib.isdf_points_fixed_rank(_ptr(phi), _ptr(dphi), _ptr(w), n_g, n_orb, n_ch_phi,
                                    n_ch_grad, _ptr(piv), ctypes.byref(out), _ptr(ws), ws.numel(),
                                    _stream())
    C.check("isdf_points_fixed_rank", st, allow=(C.ISDF_E_RANK,) if allow_rank else ())
    return piv[:out.value]


def isdf_fit(phi, dphi, pivots, jitter_init: float = 0.0, jitter_growth: float = 0.0,
             max_jitter_tries: int = 0, fit_mode: int = 0):
    """xi [n_mu][n_g], xi~ [3][n_mu][n_g] and the jitter per system.  The
    jitter policy (Sec. IV.B): 0 selects the library defaults (1e-14 of the
    largest diagonal, x10 per retry, 8 retries); max_jitter_tries < 0 allows none.
    fit_mode 1 runs the right-hand sides and the solves as FP64 products
    emulated on the tensor cores."""
    lib = C.load()
    dev = phi.device
    n_orb, n_g = _orbital_planes(phi, dphi, lambda _: (pivots, torch.int32, "pivots", (None,)))
    n_mu = pivots.numel()
    xi = torch.empty((n_mu, n_g), dtype=f64, device=dev)
    xig = torch.empty((3, n_mu, n_g), dtype=f64, device=dev)
    jit = (ctypes.c_double * 4)()
    ws = _ws(lib.isdf_fit_workspace_mode(n_g, n_orb, n_mu, int(fit_mode)), dev)
    opt = options(jitter_init=jitter_init, jitter_growth=jitter_growth,
                  max_jitter_tries=max_jitter_tries, fit_mode=fit_mode)
    C.check("isdf_fit", lib.isdf_fit(_ptr(phi), _ptr(dphi), n_g, n_orb, _ptr(pivots), n_mu,
                                     _ptr(xi), _ptr(xig), jit, ctypes.byref(opt), _ptr(ws),
                                     ws.numel(), _stream()))
    return xi, xig, list(jit)


def isdf_dgemm_emulated(A, B, alpha: float = 1.0, out=None):
    """alpha A B, added in place to `out` when given, with the FP64 products
    emulated on the tensor cores; A [M][K], B [K][N] FP64."""
    lib = C.load()
    M, K = _dims(A, "A", 2)
    N = _shape(B, "B", (K, None))[1]
    specs = [(A, f64, "A", None), (B, f64, "B", None)]
    beta = 0.0
    if out is not None:
        specs.append((out, f64, "out", (M, N)))
        beta = 1.0
    _reqs(*specs)
    if out is None:
        out = torch.empty((M, N), dtype=f64, device=A.device)
    ws = _ws(lib.isdf_dgemm_emulated_workspace(M, N, K), A.device)
    C.check("isdf_dgemm_emulated", lib.isdf_dgemm_emulated(
        M, N, K, _ptr(A), K, _ptr(B), N, float(alpha), beta, _ptr(out), N, _ptr(ws), ws.numel(),
        _stream()))
    return out


def isdf_gather_pivots(phi, dphi, pivots):
    """phi_p(r_mu) [n_mu][n_orb] and d_c phi_p(r_mu) [3][n_mu][n_orb] at the
    pivots: the factors of the pivot tensors C^p_q(r_mu) of Eq. isdf-rho."""
    lib = C.load()
    n_orb, n_g = _orbital_planes(phi, dphi, lambda _: (pivots, torch.int32, "pivots", (None,)))
    n_mu = pivots.numel()
    phiP = torch.empty((n_mu, n_orb), dtype=f64, device=phi.device)
    dphiP = torch.empty((3, n_mu, n_orb), dtype=f64, device=phi.device)
    C.check("isdf_gather_pivots", lib.isdf_gather_pivots(
        _ptr(phi), _ptr(dphi), n_g, n_orb, _ptr(pivots), n_mu, _ptr(phiP), _ptr(dphiP), _stream()))
    return phiP, dphiP


def options(precision="bf16x3", kchunk: int = 0, s2_kchunk: int = 0, sync_check: bool = True,
            debug_flags: int = 0, stage_ms=None, jitter_init: float = 0.0,
            jitter_growth: float = 0.0, max_jitter_tries: int = 0,
            wait_limit_ms: int = 0, fit_mode: int = 0) -> C.IsdfOptions:
    """isdf_options for the W build and the fit; 0 selects the library defaults."""
    prec = C.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return C.IsdfOptions(prec, kchunk, s2_kchunk, int(sync_check), debug_flags, stage_ms,
                         float(jitter_init), float(jitter_growth), int(max_jitter_tries),
                         int(wait_limit_ms), int(fit_mode))


class KernelBuilder:
    """Reusable W-build call: output and workspace tensors are allocated once,
    so that repeated calls (benchmarks, CUDA graphs) allocate nothing."""

    def __init__(self, grid_xyz, w, xi, xig, jastrow: C.IsdfJastrow, precision="bf16x3",
                 g_begin: int = 0, g_end: Optional[int] = None, kchunk: int = 0,
                 s2_kchunk: int = 0, sync_check: bool = True, debug_flags: int = 0,
                 time_stages: bool = False, wait_limit_ms: int = 0):
        lib = C.load()
        n_mu, n_g = _dims(xi, "xi", 2)
        _reqs((xi, f64, "xi", None), (xig, f64, "xi_grad", (3, n_mu, n_g)),
              (grid_xyz, f64, "grid_xyz", (n_g, 3)), (w, f64, "w", (n_g,)))
        self.lib = lib
        self.dev = xi.device
        self.n_mu, self.n_g = n_mu, n_g
        self.g_begin = int(g_begin)
        self.g_end = int(self.n_g if g_end is None else g_end)
        self.args = (grid_xyz, w, xi, xig)
        self.J = jastrow
        self.stage_ms = (ctypes.c_float * 2)() if time_stages else None
        self.opt = options(precision, kchunk, s2_kchunk, sync_check, debug_flags,
                           ctypes.cast(self.stage_ms, ctypes.POINTER(ctypes.c_float))
                           if time_stages else None, wait_limit_ms=wait_limit_ms)
        n_gs = max(self.g_end - self.g_begin, 0)  # an empty slice is rejected by the library
        self.W = torch.empty((4, self.n_mu, self.n_mu), dtype=f64, device=self.dev)
        self.calG = torch.empty((4, self.n_mu, n_gs), dtype=f64, device=self.dev)
        self.ws = _ws(lib.tc_kernel_build_workspace(self.n_g, self.n_mu, self.g_begin, self.g_end,
                                                   self.opt.precision, ctypes.byref(self.J)),
                      self.dev)

    def __call__(self, allow_timeout: bool = False):
        g, w, xi, xig = self.args
        st = self.lib.tc_kernel_build(_ptr(g), _ptr(w), _ptr(xi), _ptr(xig), self.n_g, self.n_mu,
                                      self.g_begin, self.g_end, ctypes.byref(self.J),
                                      ctypes.byref(self.opt), _ptr(self.W), _ptr(self.calG),
                                      _ptr(self.ws), self.ws.numel(), _stream())
        C.check("tc_kernel_build", st, allow=(C.ISDF_E_TIMEOUT,) if allow_timeout else ())
        return st


def tc_kernel_build(grid_xyz, w, xi, xig, jastrow: C.IsdfJastrow, precision="bf16x3",
                    g_begin: int = 0, g_end: Optional[int] = None, kchunk: int = 0,
                    s2_kchunk: int = 0, stage_ms: Optional[list] = None):
    """W [4][n_mu][n_mu] (u1x, u1y, u1z, u3) and calG [4][n_mu][g_end-g_begin].
    When ``stage_ms`` is a list, the device times of stage 1 and 2 are
    appended to it (tensor-core precisions)."""
    kb = KernelBuilder(grid_xyz, w, xi, xig, jastrow, precision, g_begin, g_end, kchunk, s2_kchunk,
                       time_stages=stage_ms is not None)
    kb()
    if stage_ms is not None:
        stage_ms.append(tuple(kb.stage_ms))
    return kb.W, kb.calG


def tc_kernel_build_streamed(grid_xyz, w, xi_host, xig_host, jastrow: C.IsdfJastrow,
                             precision="bf16x3", bra: int = 16384, ket: int = 16384,
                             kchunk: int = 0):
    """W [4][n_mu][n_mu] on the device from xi [n_mu][n_g] and xi~ [3][n_mu][n_g]
    held in (pinned) host memory, streamed in bra/ket grid batches with a
    depth-one prefetch (Sec. II.D); grid_xyz and w on the device."""
    lib = C.load()
    for t, n in ((xi_host, "xi_host"), (xig_host, "xig_host")):
        if t.device.type != "cpu" or t.dtype != f64 or not t.is_contiguous():
            raise ValueError(f"{n} must be a contiguous FP64 host tensor")
    if xi_host.dim() != 2:
        raise ValueError(f"xi_host has shape {tuple(xi_host.shape)}, expected (n_mu, n_g)")
    n_mu, n_g = xi_host.shape
    if tuple(xig_host.shape) != (3, n_mu, n_g):
        raise ValueError(f"xig_host has shape {tuple(xig_host.shape)}, expected {(3, n_mu, n_g)}")
    _reqs((grid_xyz, f64, "grid_xyz", (n_g, 3)), (w, f64, "w", (n_g,)))
    dev = grid_xyz.device
    opt = options(precision, kchunk)
    W = torch.empty((4, n_mu, n_mu), dtype=f64, device=dev)
    ws = _ws(lib.tc_kernel_build_streamed_workspace(n_g, n_mu, bra, ket, opt.precision,
                                                    ctypes.byref(jastrow)), dev)
    C.check("tc_kernel_build_streamed", lib.tc_kernel_build_streamed(
        _ptr(grid_xyz), _ptr(w), ctypes.c_void_p(xi_host.data_ptr()),
        ctypes.c_void_p(xig_host.data_ptr()), n_g, n_mu, bra, ket, ctypes.byref(jastrow),
        ctypes.byref(opt), _ptr(W), _ptr(ws), ws.numel(), _stream()))
    return W


def grid_shard(n_g: int, rank: int, world: int) -> Tuple[int, int]:
    """The outer-grid slice [g_begin, g_end) of rank ``rank`` of ``world`` for a
    sharded W build (Sec. IV.C): contiguous, covering [0, n_g) once, sizes
    differing by at most one tile of 64 points.  The partial kernels of the
    slices sum to the full W (one all-reduce of 4 n_mu^2 values)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    tiles = (n_g + 63) // 64
    t0 = tiles * rank // world
    t1 = tiles * (rank + 1) // world
    return min(64 * t0, n_g), min(64 * t1, n_g)


def kernel_launches() -> int:
    """Kernels launched by libisdftc in this process so far."""
    return int(C.load().isdf_kernel_launches())


def xtc_density_contract(phi_piv, n_occ: int, xi, w, calG, n_orb_x: int = 0,
                         precision="fp64"):
    """D [n_mu][n_mu] and (n_orb_x > 0) X packed [n_orb_x(n_orb_x+1)/2][n_mu]."""
    lib = C.load()
    dev = xi.device
    n_mu, n_g = _dims(xi, "xi", 2)
    n_orb = _shape(phi_piv, "phi_piv", (n_mu, None))[1]
    if _shape(calG, "calG", (None, n_mu, n_g))[0] < 3:
        raise ValueError("calG needs its three gradient channels")
    _reqs((xi, f64, "xi", None), (phi_piv, f64, "phi_piv", None), (w, f64, "w", (n_g,)),
          (calG, f64, "calG", None))
    prec = C.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    D = torch.empty((n_mu, n_mu), dtype=f64, device=dev)
    Xp = torch.empty((n_orb_x * (n_orb_x + 1) // 2, n_mu), dtype=f64, device=dev) if n_orb_x > 0 else None
    ws = _ws(lib.xtc_density_contract_workspace(n_g, n_mu, n_orb, n_occ, n_orb_x, prec), dev)
    C.check("xtc_density_contract", lib.xtc_density_contract(
        _ptr(phi_piv), n_orb, n_occ, _ptr(xi), _ptr(w), _ptr(calG), n_g, n_mu, _ptr(D), _ptr(Xp),
        n_orb_x, prec, _ptr(ws), ws.numel(), _stream()))
    return D, Xp


def tc_energies(W, D, Xp, phi_piv, dphi_piv, n_occ: int):
    """(E_K, E_dU, E0) in Hartree from the factors (occupied block)."""
    lib = C.load()
    n_mu, n_orb = _factors(W, D, Xp, phi_piv, dphi_piv, n_occ * (n_occ + 1) // 2)
    out = (ctypes.c_double * 3)()
    ws = _ws(lib.tc_energies_workspace(n_mu, n_occ), W.device)
    C.check("tc_energies", lib.tc_energies(_ptr(W), _ptr(D), _ptr(Xp), _ptr(phi_piv), _ptr(dphi_piv),
                                           n_mu, n_orb, n_occ, out, _ptr(ws), ws.numel(), _stream()))
    return tuple(out)


def tc_two_body_panel(W, D, Xp, phi_piv, dphi_piv, pr_begin: int, pr_end: int,
                      precision="fp64", want_k: bool = True, want_du: bool = True):
    """Rows [pr_begin, pr_end) of the four-index K and DeltaU in composite form
    (row (p,r) = p n_orb + r, column (q,s)); Xp is the full packed X."""
    lib = C.load()
    n_mu, n_orb = _factors(W, D, Xp, phi_piv, dphi_piv)
    rows = pr_end - pr_begin
    prec = C.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    dev = phi_piv.device
    K = torch.empty((rows, n_orb * n_orb), dtype=f64, device=dev) if want_k else None
    U = torch.empty((rows, n_orb * n_orb), dtype=f64, device=dev) if want_du else None
    ws = _ws(lib.tc_two_body_panel_workspace(n_mu, n_orb, rows, prec), dev)
    C.check("tc_two_body_panel", lib.tc_two_body_panel(
        _ptr(W), _ptr(D), _ptr(Xp), _ptr(phi_piv), _ptr(dphi_piv), n_mu, n_orb, pr_begin, pr_end,
        prec, _ptr(K), _ptr(U), _ptr(ws), ws.numel(), _stream()))
    return K, U


def tc_xtc_one_body(W, D, Xp, phi_piv, dphi_piv, n_occ: int):
    """Delta h [n_orb][n_orb], f^xTC [n_orb][n_orb] and E0 (Eqs. xtc-deltah,
    xtc-fock, xtc-const); Xp is the full packed X."""
    lib = C.load()
    n_mu, n_orb = _factors(W, D, Xp, phi_piv, dphi_piv)
    dev = phi_piv.device
    dh = torch.empty((n_orb, n_orb), dtype=f64, device=dev)
    f = torch.empty((n_orb, n_orb), dtype=f64, device=dev)
    e0 = ctypes.c_double(0.0)
    ws = _ws(lib.tc_xtc_one_body_workspace(n_mu, n_orb), dev)
    C.check("tc_xtc_one_body", lib.tc_xtc_one_body(
        _ptr(W), _ptr(D), _ptr(Xp), _ptr(phi_piv), _ptr(dphi_piv), n_mu, n_orb, n_occ, _ptr(dh),
        _ptr(f), ctypes.byref(e0), _ptr(ws), ws.numel(), _stream()))
    return dh, f, e0.value


def tc_kernel_adjoint(grid_xyz, w, xi, xig, jastrow: C.IsdfJastrow, Wbar, precision="fp32",
                      g_begin: Optional[int] = None, g_end: Optional[int] = None):
    """dL/dtheta for L = sum_c <Wbar^c, W^c>, theta = (d, b, c_0 .. c_{K-1});
    with g_begin/g_end, W over that outer-grid slice only."""
    lib = C.load()
    n_mu, n_g = _dims(xi, "xi", 2)
    _reqs((xi, f64, "xi", None), (xig, f64, "xi_grad", (3, n_mu, n_g)),
          (grid_xyz, f64, "grid_xyz", (n_g, 3)), (w, f64, "w", (n_g,)),
          (Wbar, f64, "Wbar", (4, n_mu, n_mu)))
    prec = C.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    dtheta = torch.empty(2 + jastrow.n_terms, dtype=f64, device=xi.device)
    ws = _ws(lib.tc_kernel_adjoint_workspace(n_g, n_mu, jastrow.n_nuc, prec), xi.device)
    if g_begin is None and g_end is None:
        st = lib.tc_kernel_adjoint(
            _ptr(grid_xyz), _ptr(w), _ptr(xi), _ptr(xig), n_g, n_mu, ctypes.byref(jastrow),
            _ptr(Wbar), prec, _ptr(dtheta), _ptr(ws), ws.numel(), _stream())
    else:
        g0 = 0 if g_begin is None else int(g_begin)
        g1 = n_g if g_end is None else int(g_end)
        st = lib.tc_kernel_adjoint_range(
            _ptr(grid_xyz), _ptr(w), _ptr(xi), _ptr(xig), n_g, n_mu, g0, g1,
            ctypes.byref(jastrow), _ptr(Wbar), prec, _ptr(dtheta), _ptr(ws), ws.numel(),
            _stream())
    C.check("tc_kernel_adjoint", st)
    return dtheta


def jastrow_with_theta(template: C.IsdfJastrow, theta) -> C.IsdfJastrow:
    """Copy of a one-type correlator with theta = (d, b, c_0 .. c_{K-1})."""
    J = C.IsdfJastrow()
    ctypes.pointer(J)[0] = template
    th = [float(x) for x in theta]
    J.d = th[0]
    J.b[0] = th[1]
    for k in range(template.n_terms):
        J.coef[0][k] = th[2 + k]
    return J


class TCKernel(torch.autograd.Function):
    """W = {u1x, u1y, u1z, u3} as a differentiable function of the correlator
    parameters theta.  Forward: FP64 kernel build; backward: the adjoint
    kernel (dW/dtheta contracted with the incoming gradient), with the M
    tiles recomputed instead of stored."""

    @staticmethod
    def forward(ctx, theta, grid_xyz, w, xi, xig, template, adjoint_precision="fp32"):
        J = jastrow_with_theta(template, theta.detach().cpu().tolist())
        W, _ = tc_kernel_build(grid_xyz, w, xi, xig, J, "fp64")
        ctx.save_for_backward(grid_xyz, w, xi, xig)
        ctx.J = J
        ctx.prec = adjoint_precision
        ctx.theta_device = theta.device
        return W

    @staticmethod
    def backward(ctx, Wbar):
        grid_xyz, w, xi, xig = ctx.saved_tensors
        g = tc_kernel_adjoint(grid_xyz, w, xi, xig, ctx.J, Wbar.contiguous(), ctx.prec)
        return g.to(ctx.theta_device), None, None, None, None, None, None


def _basis(center, powers, exps, coefs, *more) -> C.IsdfBasis:
    """The isdf_basis struct over the four device arrays, checked with the
    further specs `more` (shapes first)."""
    n_bf, n_prim = _dims(exps, "exps", 2)
    _reqs((exps, f64, "exps", None), (coefs, f64, "coefs", (n_bf, n_prim)),
          (center, f64, "center", (n_bf, 3)), (powers, torch.int32, "powers", (n_bf, 3)), *more)
    return C.IsdfBasis(n_bf, n_prim, _ptr(center), _ptr(powers), _ptr(exps), _ptr(coefs))


def isdf_vmc_local_energy(basis, mo_coef, n_occ: int, walkers, jastrow: C.IsdfJastrow, charges,
                          theta=None, fd_step: float = 1e-5, grad: bool = True):
    """E_loc [n_walkers] of Eq. Eloc and, with grad, dE_loc/dtheta [P][n_walkers]
    (theta = (d, b_t, coef row-major); None = the struct's values).
    basis = (center, powers, exps, coefs) device tensors; charges host [n_nuc]."""
    if len(charges) != jastrow.n_nuc:
        raise ValueError(f"charges has {len(charges)} values for {jastrow.n_nuc} nuclei")
    lib = C.load()
    n_bf = _dims(basis[2], "exps", 2)[0]
    B = _basis(*basis, (mo_coef, f64, "mo_coef", (n_bf, None)),
               (walkers, f64, "walkers", (None, 2 * n_occ, 3)))
    dev = walkers.device
    n_walk = walkers.shape[0]
    P = lib.isdf_vmc_n_params(ctypes.byref(jastrow))
    if theta is not None:
        _req(theta, f64, "theta")
        if theta.numel() != P:
            raise ValueError(f"theta needs {P} values")
    Z = (ctypes.c_double * max(1, jastrow.n_nuc))(*[float(z) for z in charges])
    E = torch.empty(n_walk, dtype=f64, device=dev)
    dE = torch.empty((P, n_walk), dtype=f64, device=dev) if grad else None
    ws = _ws(lib.isdf_vmc_local_energy_workspace(B.n_bf, n_occ, n_walk, ctypes.byref(jastrow)), dev)
    C.check("isdf_vmc_local_energy", lib.isdf_vmc_local_energy(
        ctypes.byref(B), _ptr(mo_coef), mo_coef.shape[1], n_occ, _ptr(walkers), n_walk,
        ctypes.byref(jastrow), ctypes.cast(Z, ctypes.c_void_p), _ptr(theta), float(fd_step),
        _ptr(E), _ptr(dE), _ptr(ws), ws.numel(), _stream()))
    return (E, dE) if grad else E


def isdf_vmc_sample(basis, mo_coef, n_occ: int, walkers, normals, uniforms, sigma: float) -> int:
    """Metropolis sweeps on |Phi_0|^2, walkers moved in place; returns the
    number of accepted moves (synchronises)."""
    lib = C.load()
    n_bf = _dims(basis[2], "exps", 2)[0]
    n_w = _shape(walkers, "walkers", (None, 2 * n_occ, 3))[0]
    n_steps = _shape(uniforms, "uniforms", (None, 2 * n_occ, n_w))[0]
    B = _basis(*basis, (mo_coef, f64, "mo_coef", (n_bf, None)), (walkers, f64, "walkers", None),
               (uniforms, f64, "uniforms", None),
               (normals, f64, "normals", (n_steps, 2 * n_occ, n_w, 3)))
    acc = torch.zeros(1, dtype=torch.int64, device=walkers.device)
    C.check("isdf_vmc_sample", lib.isdf_vmc_sample(
        ctypes.byref(B), _ptr(mo_coef), mo_coef.shape[1], n_occ, _ptr(walkers), walkers.shape[0],
        _ptr(normals), _ptr(uniforms), n_steps, float(sigma), _ptr(acc), _stream()))
    return int(acc.item())


def isdf_vmc_gn_step(E, dE, lam: float, eta: float, theta=None):
    """Gauss-Newton step of Eq. gn: returns (step [P], stats [4] = clipped
    mean, variance, raw mean, mean absolute deviation); theta += step in place
    when given."""
    lib = C.load()
    n_w = _dims(E, "E", 1)[0]
    P = _shape(dE, "dE", (None, n_w))[0]
    _reqs((E, f64, "E", None), (dE, f64, "dE", None),
          *([(theta, f64, "theta", (P,))] if theta is not None else []))
    step = torch.empty(P, dtype=f64, device=E.device)
    stats = torch.empty(4, dtype=f64, device=E.device)
    ws = _ws(lib.isdf_vmc_gn_step_workspace(n_w, P), E.device)
    C.check("isdf_vmc_gn_step", lib.isdf_vmc_gn_step(
        _ptr(E), _ptr(dE), n_w, P, float(lam), float(eta), _ptr(theta), _ptr(step), _ptr(stats),
        _ptr(ws), ws.numel(), _stream()))
    return step, stats


def isdf_vmc_objective(E):
    """stats [4] = (clipped mean, clipped variance, raw mean, mean absolute
    deviation) of Eq. var-loss."""
    lib = C.load()
    _req(E, f64, "E")
    stats = torch.empty(4, dtype=f64, device=E.device)
    C.check("isdf_vmc_objective", lib.isdf_vmc_objective(_ptr(E), E.numel(), _ptr(stats), _stream()))
    return stats


class VmcOptimizer:
    """Gauss-Newton iterations of Eq. gn (reference-variance protocol) with an
    adaptive Tikhonov shift: a step is kept only when the clipped variance at
    the new theta, on the same walkers, is lower than at the current theta
    (then lam /= 3); otherwise theta stays and lam *= 10.  theta (device [P])
    is updated in place; the walkers may be moved between steps (a fresh
    sample of |Phi_0|^2 per step)."""

    def __init__(self, basis, mo_coef, n_occ: int, walkers, jastrow: C.IsdfJastrow, charges,
                 theta, lam: float = 1e-3, eta: float = 0.5, fd_step: float = 1e-5,
                 lam_min: float = 1e-8, lam_max: float = 1e6):
        self.args = (basis, mo_coef, n_occ, walkers, jastrow, charges)
        self.theta, self.lam, self.eta, self.h = theta, lam, eta, fd_step
        self.lam_min, self.lam_max = lam_min, lam_max
        E = isdf_vmc_local_energy(*self.args, theta, fd_step, grad=False)
        self.var = float(isdf_vmc_objective(E)[1])

    def step(self):
        """One iteration on the current walkers; returns (variance, lam, accepted)."""
        E, dE = isdf_vmc_local_energy(*self.args, self.theta, self.h)
        trial = self.theta.clone()
        _, stats = isdf_vmc_gn_step(E, dE, self.lam, self.eta, theta=trial)
        cur = float(stats[1])
        Et = isdf_vmc_local_energy(*self.args, trial, self.h, grad=False)
        vt = float(isdf_vmc_objective(Et)[1])
        ok = vt < cur
        if ok:
            self.theta.copy_(trial)
            self.var = vt
            self.lam = max(self.lam / 3.0, self.lam_min)
        else:
            self.var = cur
            self.lam = min(self.lam * 10.0, self.lam_max)
        return self.var, self.lam, ok


def isdf_vmc_polyak(theta, avg, k: int):
    """avg += (theta - avg) / k in place (the k-th Polyak-Ruppert iterate; at
    k = 1 avg becomes theta whatever it held)."""
    if avg.numel() != theta.numel():
        raise ValueError(f"avg has {avg.numel()} values, theta {theta.numel()}")
    lib = C.load()
    _req(theta, f64, "theta"); _req(avg, f64, "avg")
    C.check("isdf_vmc_polyak", lib.isdf_vmc_polyak(_ptr(theta), _ptr(avg), theta.numel(), int(k),
                                                   _stream()))
    return avg


def vmc_schedule(basis, mo_coef, n_occ: int, walkers, jastrow: C.IsdfJastrow, charges, theta,
                 n_warm: int, n_refine: int, window: int, sweeps: int, sigma: float,
                 generator=None, **kw):
    """A warm-up / refinement run of the reference-variance optimisation
    (Sec. II.C): every step continues the walkers' Metropolis chains on
    |Phi_0|^2 for `sweeps` sweeps (random numbers drawn on the device from
    `generator`), then takes one VmcOptimizer step on them; the production
    parameters are the Polyak-Ruppert average of theta over the last `window`
    refinement steps.  theta is updated in place; returns (theta_avg, history
    of (variance, lam, accepted, acceptance ratio))."""
    if not 1 <= window <= n_refine:
        raise ValueError("need 1 <= window <= n_refine")
    N = 2 * n_occ
    n_w = walkers.shape[0]
    opt = VmcOptimizer(basis, mo_coef, n_occ, walkers, jastrow, charges, theta, **kw)
    avg = torch.empty_like(theta)
    hist = []
    for s in range(n_warm + n_refine):
        normals = torch.randn((sweeps, N, n_w, 3), dtype=f64, device=walkers.device,
                              generator=generator)
        uniforms = torch.rand((sweeps, N, n_w), dtype=f64, device=walkers.device,
                              generator=generator)
        acc = isdf_vmc_sample(basis, mo_coef, n_occ, walkers, normals, uniforms, sigma)
        var, lam, ok = opt.step()
        hist.append((var, lam, ok, acc / float(sweeps * N * n_w)))
        k = s - (n_warm + n_refine - window) + 1
        if k >= 1:
            isdf_vmc_polyak(theta, avg, k)
    return avg, hist


def vmc_optimize(basis, mo_coef, n_occ: int, walkers, jastrow: C.IsdfJastrow, charges, theta,
                 n_iter: int, **kw):
    """n_iter iterations of VmcOptimizer; returns their (variance, lam,
    accepted) history."""
    opt = VmcOptimizer(basis, mo_coef, n_occ, walkers, jastrow, charges, theta, **kw)
    return [opt.step() for _ in range(n_iter)]
