"""GB300-native level-set / adjoint LLG solver (arXiv 2411.19109 hot path).

The compute path is the CUDA library built from csrc/ (include/llg.h is its
C ABI); this package holds its build script and the ctypes / torch binding.
"""
from .llg import (LLG_CKPT_BINOMIAL, LLG_CKPT_PERIODIC, LLG_CKPT_STORE_ALL, LLG_FP32, LLG_FP64, LLG_J_ENERGY_AREA,
                  LLG_J_PORT, LLG_J_SPECTRAL, LLG_J_CURVE, LLGError, Solver, levelset_step, llg_adjoint, llg_create, llg_destroy,
                  llg_field, llg_field_noalloc, llg_forward, llg_function, llg_kernel_time, llg_launch_count, llg_last_error,
                  llg_padded_extents, llg_query, llg_schedule, load, llg_rbf_workspace_bytes, llg_rbf_phi,
                  llg_rbf_grad, llg_adam_step, llg_fp64_fma_rate, llg_adaptive_steps, make_rbf,
                  llg_launch_config, LLG_SPEC_WORKING, LLG_SPEC_DFLOAT, LLG_TUNE_DEFAULT, LLG_TUNE_MEASURE,
                  LLG_TUNE_GIVEN, LLG_RECORD_STAGES, LLG_RECORD_STATES)

__all__ = ["Solver", "LLGError", "load", "llg_create", "llg_forward", "llg_adjoint", "levelset_step",
           "llg_field", "llg_field_noalloc", "llg_query", "llg_launch_count", "llg_kernel_time", "llg_last_error", "llg_destroy",
           "llg_schedule", "llg_padded_extents", "llg_function", "llg_rbf_workspace_bytes", "llg_rbf_phi",
           "llg_rbf_grad", "llg_adam_step", "llg_fp64_fma_rate", "llg_adaptive_steps", "make_rbf", "LLG_FP32", "LLG_FP64",
           "LLG_CKPT_BINOMIAL", "LLG_CKPT_PERIODIC", "LLG_CKPT_STORE_ALL", "LLG_J_PORT", "LLG_J_ENERGY_AREA",
           "LLG_J_SPECTRAL", "LLG_J_CURVE", "llg_launch_config", "LLG_SPEC_WORKING", "LLG_SPEC_DFLOAT",
           "LLG_TUNE_DEFAULT", "LLG_TUNE_MEASURE", "LLG_TUNE_GIVEN", "LLG_RECORD_STAGES", "LLG_RECORD_STATES"]
