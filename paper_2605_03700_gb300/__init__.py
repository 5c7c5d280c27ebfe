"""GB300-native CF-DQMC sweep for the LLL-projected SO(5) model (arXiv:2605.03700).

The compute path is libqmc.so (hand-written CUDA for sm_103a behind a C ABI,
include/qmc.h); ``qmc`` is its ctypes binding.
"""
from .qmc import (QMC_DRIFT_EXACT, QMC_DRIFT_FIRST, QMC_SLICE_SHARED, QMC_SLICE_INDEP, QMC_NOBS, QMC_NTRACE, QMC_SPHERE, QMC_TORUS,
                  OBS_NAMES, Chain, Group, Net, QMCError,
                  lib, qmc_default_opts, qmc_launch_count, qmc_profile_gemm,
                  qmc_ratio_update, qmc_tau_int, qmc_gemm_tile, qmc_peak_fma, qmc_cgemm, qmc_profile_tensor,
                  qmc_eigh, qmc_udv)

__all__ = ["Chain", "Group", "Net", "QMCError", "QMC_TORUS", "QMC_SPHERE", "QMC_NOBS", "QMC_NTRACE",
           "QMC_DRIFT_EXACT", "QMC_DRIFT_FIRST", "QMC_SLICE_SHARED", "QMC_SLICE_INDEP",
           "OBS_NAMES", "lib", "qmc_default_opts", "qmc_tau_int", "qmc_launch_count",
           "qmc_profile_gemm", "qmc_ratio_update", "qmc_gemm_tile", "qmc_peak_fma", "qmc_cgemm", "qmc_profile_tensor",
           "qmc_eigh", "qmc_udv"]
