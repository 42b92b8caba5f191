"""GB300 (sm_103a) implementation of the PIRMCut IRLS hot path.

The compute path is ``libpirmcut.so`` (CUDA kernels behind the C ABI of
``include/pirmcut.h``); :mod:`paper_1501_03105_gb300.binding` is its ctypes
binding and :mod:`paper_1501_03105_gb300.build` compiles it.
"""
from .binding import (  # noqa: F401
    Options,
    StepInfo,
    PirmcutError,
    Solver,
    Batch,
    pirmcut_batch_create,
    pirmcut_batch_solve,
    pirmcut_batch_cut,
    pirmcut_batch_get_x,
    pirmcut_batch_info,
    pirmcut_batch_kernel_launches,
    pirmcut_batch_destroy,
    pirmcut_default_options,
    pirmcut_create,
    pirmcut_initial,
    pirmcut_irls_step,
    pirmcut_solve,
    pirmcut_cut,
    pirmcut_cut_two_level,
    pirmcut_get_x,
    pirmcut_set_x,
    pirmcut_update_weights,
    pirmcut_problem_size,
    pirmcut_kernel_launches,
    pirmcut_mlp_enable,
    pirmcut_mlp_configure,
    pirmcut_mlp_predict,
    pirmcut_mlp_weights,
    pirmcut_mlp_stats,
    pirmcut_mlp_features,
    MlpInfo,
    pirmcut_time_spmv,
    pirmcut_spmv_timing,
    pirmcut_last_error,
    pirmcut_destroy,
)
