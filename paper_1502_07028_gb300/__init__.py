"""GB300-native parallelised traveling-cluster Monte Carlo (PTCA hot path).

The compute lives in libptca.so (hand-written CUDA for sm_103a behind the C
ABI in include/ptca.h); ``ptca`` is its ctypes binding.
"""
from .ptca import (Config, Context, PtcaError, FP64, MIXED, SCHEDULE_TILED, SCHEDULE_BLOCK, PROPOSAL_SPHERE,
                   PROPOSAL_CONE, ptca_init, ptca_destroy, ptca_set_T, ptca_set_mu, ptca_get_spins, ptca_set_spins,
                   ptca_dims, ptca_build_clusters, ptca_cluster_eigvals, ptca_free_energy, ptca_sweep,
                   ptca_sweep_record, ptca_observables, ptca_schedule, ptca_version, ptca_sweep_noalloc, ptca_set_pipeline, ptca_set_resolve_margin, ptca_set_checker, ptca_checker_read, ptca_set_launch_config,
                   ptca_get_launch_config, ptca_autotune, LaunchConfig, ptca_set_kernel_timing, ptca_kernel_times,
                   KernelTimes, ptca_stage_split, ptca_full_spectrum, PIPELINE_OVERLAP, MODEL_DOUBLE_EXCHANGE, MODEL_HUBBARD_MF, MODEL_HOLSTEIN,
                   ptca_surrogate_param_count, ptca_surrogate_init, ptca_surrogate_get_params,
                   ptca_surrogate_set_params, ptca_surrogate_collect, ptca_surrogate_train, ptca_surrogate_grad,
                   ptca_surrogate_predict, ptca_surrogate_enable,
                   ptca_selftest_barrier_timeout, PIPELINE_STAGES, PIPELINE_PERSISTENT, PIPELINE_GRAPH, lib,
                   library_path)

__all__ = [n for n in dir() if not n.startswith("_")]
