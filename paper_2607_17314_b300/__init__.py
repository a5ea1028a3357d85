"""B300-native (sm_103a) ISDF-xTC transcorrelated kernel build.

The CUDA library ``libisdftc.so`` (C ABI in ``include/isdftc.h``) computes
every step; this package holds its ctypes binding (``_capi``), a torch-facing
front end with the same names (``api``) and the step-by-step driver of the
whole path (``pipeline``).
"""
from . import _capi  # noqa: F401
from .api import (KernelBuilder, isdf_eval_orbitals, isdf_fit, isdf_gather_pivots,  # noqa: F401
                  isdf_points, isdf_points_fixed_rank, jastrow_from, jastrow_struct,
                  tc_energies, tc_kernel_build, tc_kernel_build_streamed,
                  isdf_vmc_gn_step, isdf_vmc_local_energy, isdf_vmc_objective, isdf_vmc_polyak,
                  isdf_vmc_sample, vmc_optimize, vmc_schedule,
                  xtc_density_contract)
