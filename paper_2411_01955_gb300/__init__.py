"""GB300 (sm_103a) hot path of annealed plug-and-play HQS reconstruction for
multicoil non-Cartesian MRI (arXiv 2411.01955): gridding NUFFT, Toeplitz A^H A,
preconditioned CG data consistency and the HQS outer loop.

This module is a thin ctypes binding of the C ABI in include/hqs.h: it only
marshals torch CUDA tensors (device memory) and the current CUDA stream into
the library calls.  Every step of the path runs in the library's kernels; if
the compiled library is missing the import of any entry point fails loudly.
"""
from ._lib import (  # noqa: F401
    HQS_OK, HQS_ERR_INVALID_ARG, HQS_ERR_OOM, HQS_ERR_NOT_CONVERGED, HQS_ERR_BREAKDOWN,
    HQS_ERR_TIMEOUT, HQS_ERR_CALLBACK, HQS_ERR_CUDA, HQS_ERR_UNSUPPORTED,
    HQS_PREC_FP32, HQS_PREC_BF16X3, HQS_PREC_FP16X3,
    HQS_PRECOND_NONE, HQS_PRECOND_DC, HQS_PRECOND_LEARNED,
    HQS_SOLVE_PLAIN, HQS_SOLVE_FUSED, HQS_SOLVE_X0_ZERO, HQS_MAX_ITERS,
    HqsError, Plan, SolveInfo, library, library_path,
    plan_create, forward, adjoint, adjoint_axpy, toeplitz_normal, precond_apply, dc_solve,
    last_solve_info, hqs_run, gaussian_denoise, power_iteration, status_string,
    debug_phase_trace, plan_set_tuning, precond_apply_noalloc,
    Net, plan_set_net, learned_precond_apply, Batch, plan_retile, toeplitz_stage, pgd_run, estimate_smaps, HQS_TUNE_SPREAD_TILE, HQS_TUNE_FUSED_GRID, HQS_TUNE_PC_LINES,
    HQS_TUNE_DEBUG_BARRIER_SKIP,
    Plan3d, plan3d_create, forward3d, adjoint3d, toeplitz_normal3d, plan3d_khat, dc_solve3d, precond_apply3d, gaussian_denoise3d, hqs_run3d,
)
