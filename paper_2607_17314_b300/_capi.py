"""ctypes declarations of the libisdftc C ABI (include/isdftc.h).

Argument marshalling only: every computation runs in the CUDA library.  The
library is loaded from this package directory; importing fails loudly when
it has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libisdftc.so")

ISDF_OK, ISDF_E_ARG, ISDF_E_NOT_PD, ISDF_E_RANK, ISDF_E_NONFINITE, ISDF_E_TIMEOUT, \
    ISDF_E_CUDA, ISDF_E_UNSUPPORTED = range(8)
STATUS_NAMES = ["ISDF_OK", "ISDF_E_ARG", "ISDF_E_NOT_PD", "ISDF_E_RANK", "ISDF_E_NONFINITE",
                "ISDF_E_TIMEOUT", "ISDF_E_CUDA", "ISDF_E_UNSUPPORTED"]

ISDF_PREC_FP64, ISDF_PREC_BF16X3, ISDF_PREC_BF16X6, ISDF_PREC_FP32, ISDF_PREC_TF32X3 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": ISDF_PREC_FP64, "bf16x3": ISDF_PREC_BF16X3, "bf16x6": ISDF_PREC_BF16X6,
              "fp32": ISDF_PREC_FP32, "tf32x3": ISDF_PREC_TF32X3}

ISDF_MAX_NUC, ISDF_MAX_TYPES, ISDF_MAX_TERMS = 64, 4, 32

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
SZ = ctypes.c_size_t
INT = ctypes.c_int


class IsdfBasis(ctypes.Structure):
    """ctypes mirror of isdf_basis (device pointers to the contracted Gaussians)."""
    _fields_ = [("n_bf", I32), ("n_prim", I32), ("center", P), ("powers", P), ("exps", P),
                ("coefs", P)]


class IsdfJastrow(ctypes.Structure):
    """ctypes mirror of isdf_jastrow (Boys-Handy correlator, Eqs. bh-scaled, bh-u)."""
    _fields_ = [("n_nuc", I32), ("n_types", I32), ("n_terms", I32), ("cusp", I32),
                ("d", ctypes.c_double),
                ("nuc_xyz", (ctypes.c_double * 3) * ISDF_MAX_NUC),
                ("nuc_type", I32 * ISDF_MAX_NUC),
                ("b", ctypes.c_double * ISDF_MAX_TYPES),
                ("mno", (I32 * 3) * ISDF_MAX_TERMS),
                ("coef", (ctypes.c_double * ISDF_MAX_TERMS) * ISDF_MAX_TYPES),
                ("chi_a", ctypes.c_double * ISDF_MAX_TYPES),
                ("chi_b", ctypes.c_double * ISDF_MAX_TYPES),
                ("n_elec", I32)]


class IsdfOptions(ctypes.Structure):
    """ctypes mirror of isdf_options (precision, fold intervals, checks, timing,
    jitter policy of the fit, wait limit)."""
    _fields_ = [("precision", I32), ("kchunk", I32), ("s2_kchunk", I32), ("sync_check", I32),
                ("debug_flags", I32), ("stage_ms", ctypes.POINTER(ctypes.c_float)),
                ("jitter_init", ctypes.c_double), ("jitter_growth", ctypes.c_double),
                ("max_jitter_tries", I32), ("wait_limit_ms", I32), ("fit_mode", I32)]


# name -> (restype, argtypes)
SIGNATURES = {
    "isdf_last_error": (ctypes.c_char_p, []),
    "isdf_abi_version": (INT, []),
    "isdf_kernel_launches": (ctypes.c_uint64, []),
    "isdf_eval_orbitals_workspace": (SZ, [INT, I64]),
    "isdf_eval_orbitals": (INT, [ctypes.POINTER(IsdfBasis), P, INT, P, I64, P, P, P, SZ, P]),
    "isdf_eval_orbitals_workspace_mode": (SZ, [INT, I64, INT, INT]),
    "isdf_eval_orbitals_mode": (INT, [ctypes.POINTER(IsdfBasis), P, INT, P, I64, P, P, INT, P, SZ,
                                      P]),
    "isdf_points_workspace": (SZ, [I64, INT]),
    "isdf_points": (INT, [P, P, P, I64, INT, INT, INT, P, ctypes.POINTER(INT), P, SZ, P]),
    "isdf_points_fixed_rank_workspace": (SZ, [I64, INT, INT]),
    "isdf_points_fixed_rank": (INT, [P, P, P, I64, INT, INT, INT, P, ctypes.POINTER(INT), P, SZ,
                                     P]),
    "isdf_fit_workspace": (SZ, [I64, INT, INT]),
    "isdf_fit_workspace_mode": (SZ, [I64, INT, INT, INT]),
    "isdf_dgemm_emulated_workspace": (SZ, [I64, I64, I64]),
    "isdf_dgemm_emulated": (INT, [I64, I64, I64, P, I64, P, I64, ctypes.c_double, ctypes.c_double,
                                  P, I64, P, SZ, P]),
    "isdf_fit": (INT, [P, P, I64, INT, P, INT, P, P, P, P, P, SZ, P]),
    "tc_kernel_build_streamed_workspace": (SZ, [I64, INT, I64, I64, INT, P]),
    "tc_kernel_build_streamed": (INT, [P, P, P, P, I64, INT, I64, I64, P, P, P, P, SZ, P]),
    "isdf_gather_pivots": (INT, [P, P, I64, INT, P, INT, P, P, P]),
    "tc_kernel_build_workspace": (SZ, [I64, INT, I64, I64, INT, ctypes.POINTER(IsdfJastrow)]),
    "tc_kernel_build": (INT, [P, P, P, P, I64, INT, I64, I64, ctypes.POINTER(IsdfJastrow),
                              ctypes.POINTER(IsdfOptions), P, P, P, SZ, P]),
    "tc_kernel_adjoint_workspace": (SZ, [I64, INT, INT, INT]),
    "tc_kernel_adjoint": (INT, [P, P, P, P, I64, INT, ctypes.POINTER(IsdfJastrow), P, INT, P, P,
                                SZ, P]),
    "tc_kernel_adjoint_range": (INT, [P, P, P, P, I64, INT, I64, I64, ctypes.POINTER(IsdfJastrow),
                                      P, INT, P, P, SZ, P]),
    "isdf_mlp_n_params": (INT, []),
    "isdf_mlp_features": (INT, [P, P, P, P, I64, INT, P, INT, P, P]),
    "isdf_mlp_forward": (INT, [P, P, I64, P, P]),
    "isdf_mlp_backward": (INT, [P, P, P, I64, ctypes.c_float, I64, P, P, P]),
    "isdf_mlp_adam": (INT, [P, P, P, P, INT, ctypes.c_float, P]),
    "isdf_mlp_topk": (INT, [P, I64, INT, P, P]),
    "isdf_points_restricted_workspace": (SZ, [INT, INT, INT]),
    "isdf_points_restricted": (INT, [P, P, P, I64, INT, P, INT, INT, P, ctypes.POINTER(INT), P,
                                     SZ, P]),
    "isdf_fit_error_workspace": (SZ, [I64, INT, INT]),
    "isdf_fit_error": (INT, [P, P, I64, INT, P, INT, ctypes.POINTER(ctypes.c_double), P, SZ, P]),
    "xtc_density_contract_workspace": (SZ, [I64, INT, INT, INT, INT, INT]),
    "xtc_density_contract": (INT, [P, INT, INT, P, P, P, I64, INT, P, P, INT, INT, P, SZ, P]),
    "tc_energies_workspace": (SZ, [INT, INT]),
    "tc_energies": (INT, [P, P, P, P, P, INT, INT, INT, P, P, SZ, P]),
    "tc_energies_noalloc": (INT, [P, P, P, P, P, INT, INT, INT, P, P]),
    "tc_two_body_panel_workspace": (SZ, [INT, INT, I64, INT]),
    "tc_two_body_panel": (INT, [P, P, P, P, P, INT, INT, I64, I64, INT, P, P, P, SZ, P]),
    "tc_xtc_one_body_workspace": (SZ, [INT, INT]),
    "tc_xtc_one_body": (INT, [P, P, P, P, P, INT, INT, INT, P, P,
                              ctypes.POINTER(ctypes.c_double), P, SZ, P]),
    "isdf_vmc_n_params": (INT, [ctypes.POINTER(IsdfJastrow)]),
    "isdf_vmc_local_energy_workspace": (SZ, [INT, INT, I64, ctypes.POINTER(IsdfJastrow)]),
    "isdf_vmc_local_energy": (INT, [ctypes.POINTER(IsdfBasis), P, INT, INT, P, I64,
                                    ctypes.POINTER(IsdfJastrow), P, P, ctypes.c_double, P, P,
                                    P, SZ, P]),
    "isdf_vmc_sample": (INT, [ctypes.POINTER(IsdfBasis), P, INT, INT, P, I64, P, P, INT,
                              ctypes.c_double, P, P]),
    "isdf_vmc_gn_step_workspace": (SZ, [I64, INT]),
    "isdf_vmc_objective": (INT, [P, I64, P, P]),
    "isdf_vmc_polyak": (INT, [P, P, INT, I64, P]),
    "isdf_vmc_gn_step": (INT, [P, P, I64, INT, ctypes.c_double, ctypes.c_double, P, P, P, P, SZ,
                               P]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load libisdftc.so (built in place by ``paper_2607_17314_b300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2607_17314_b300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class IsdfError(RuntimeError):
    """A libisdftc call returned a failure status; ``status`` holds it."""

    def __init__(self, func: str, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{func}: {name}: {msg}")


def check(func: str, status: int, allow=()):
    """Raise IsdfError with the library's message unless status is ISDF_OK or in
    ``allow``; return the status."""
    if status != ISDF_OK and status not in allow:
        raise IsdfError(func, status, load().isdf_last_error().decode(errors="replace"))
    return status
