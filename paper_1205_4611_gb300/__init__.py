"""GB300-native (sm_103a) adaptive 2-D fast multipole method for the
complex-log potential (Goude & Engblom, arXiv:1205.4611).

The compute path is the C-ABI library libgbfmm.so (include/gbfmm.h); this
package holds its build script and a thin ctypes binding with the same names.
"""
from .binding import (  # noqa: F401
    FMM_ERR_ARG, FMM_ERR_CUDA, FMM_ERR_NOMEM, FMM_ERR_NONFINITE, FMM_ERR_TIMEOUT, FMM_LEVELS_CAP,
    FMM_LEVELS_EQ, FMM_KERNEL_HARMONIC, FMM_KERNEL_LOG, FMM_OK, FMM_PREC_FP64, FMM_PREC_MIXED, FmmError, FmmTree, fmm_build_tree,
    fmm_default_options, fmm_evaluate, fmm_evaluate_batched, fmm_get_timings, fmm_last_error,
    fmm_launch_count, fmm_build_batched, fmm_set_graph, fmm_direct_noalloc,
    fmm_options, fmm_set_timing, fmm_solve_host, fmm_tree_export, fmm_tree_export_shortcut,
    fmm_tree_export_geometry, fmm_autotune_leaf,
    fmm_tree_info, fmm_tree_sync, fmm_memory_info, fmm_debug_inject, FMM_INJECT_ALLOC_FAILURE,
    FMM_INJECT_STATUS, fmm_autotune,
    load,
)
