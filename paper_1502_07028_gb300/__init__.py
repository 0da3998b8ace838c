"""GB300-native parallelised traveling-cluster Monte Carlo (PTCA hot path).

The compute lives in libptca.so (hand-written CUDA for sm_103a behind the C
ABI in include/ptca.h); ``ptca`` is its ctypes binding.
"""
from .ptca import (
    FP64, MIXED, MODEL_DOUBLE_EXCHANGE, MODEL_HOLSTEIN, MODEL_HUBBARD_MF, PIPELINE_GRAPH, PIPELINE_OVERLAP,
    PIPELINE_PERSISTENT, PIPELINE_STAGES, PROPOSAL_CONE, PROPOSAL_SPHERE, REDUCTION_ROWS, REDUCTION_SHARED, REDUCTION_TILED,
    SCHEDULE_BLOCK, SCHEDULE_TILED,
    Config, Context, KernelTimes, LaunchConfig, PtcaError, lib, library_path,
    ptca_autotune, ptca_build_clusters, ptca_checker_read, ptca_cluster_eigvals, ptca_destroy, ptca_dims,
    ptca_flush, ptca_free_energy, ptca_full_spectrum, ptca_get_launch_config, ptca_get_sites, ptca_get_spins, ptca_init,
    ptca_kernel_times,
    ptca_last_error, ptca_observables, ptca_schedule, ptca_selftest_barrier_timeout, ptca_set_checker,
    ptca_set_kernel_timing, ptca_set_launch_config, ptca_set_mu, ptca_set_pipeline, ptca_set_resolve_margin,
    ptca_set_sites, ptca_set_spins, ptca_set_T, ptca_stage_run, ptca_stage_split, ptca_surrogate_collect,
    ptca_surrogate_enable,
    ptca_surrogate_get_params, ptca_surrogate_grad, ptca_surrogate_init, ptca_surrogate_param_count,
    ptca_surrogate_predict, ptca_surrogate_set_params, ptca_surrogate_train, ptca_sweep, ptca_sweep_noalloc,
    ptca_sweep_record, ptca_version,
)

__all__ = [n for n in dir() if not n.startswith("_")]
