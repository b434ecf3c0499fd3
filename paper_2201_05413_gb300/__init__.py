"""GB300-native (sm_103a) Jacobi-PCG solver for FEM discretisations of the
Laplace equation: device assembly, SELL-C-sigma SpMV/SpMM, fused PCG kernels,
mixed-precision iterative refinement, batched and served solves.

The compute path is the CUDA library ``libgbpcg.so`` (C ABI in
``include/gbpcg.h``); this package only marshals arguments to it.
"""
from . import gbpcg
from .api import (FemSystem, Sell, Server, autotune, autotune_rhs_width, batched_kernel_times, pcg_solve_batched,
                  solve_multi, wait_selftest, grid_wait_selftest)
from .gbpcg import (GB_BF16_IR, GB_BF16_RU, GB_BICGSTAB, GB_CG, GB_F32_IR, GB_F32_RU, GB_F64, GB_PC_BLOCK_JACOBI,
                    GB_PC_JACOBI,
                    GB_VAL_BF16, GB_VAL_F32, GB_VAL_F64, GbError, load)

__all__ = ["FemSystem", "Sell", "Server", "autotune", "autotune_rhs_width", "batched_kernel_times", "pcg_solve_batched",
           "solve_multi", "wait_selftest", "grid_wait_selftest", "GbError", "load", "gbpcg", "GB_F64",
           "GB_F32_IR", "GB_BF16_IR", "GB_F32_RU", "GB_BF16_RU", "GB_VAL_F64", "GB_VAL_F32", "GB_VAL_BF16",
           "GB_PC_JACOBI", "GB_PC_BLOCK_JACOBI", "GB_CG", "GB_BICGSTAB"]
