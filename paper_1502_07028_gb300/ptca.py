"""Thin ctypes binding of libptca.so (C ABI declared in include/ptca.h).

Argument marshalling only: every step of the traveling-cluster hot path runs
in the library's CUDA kernels.  Torch tensors supply device memory and the
current CUDA stream; their ``data_ptr()`` is passed as a plain pointer.
There is no CPU fallback: if the library is missing or no GPU is usable the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from collections import namedtuple
from dataclasses import dataclass

from . import _build

PTCA_OK = 0
STATUS = {0: "PTCA_OK", 1: "PTCA_ERR_INVALID", 2: "PTCA_ERR_CUDA", 3: "PTCA_ERR_OOM",
          4: "PTCA_ERR_TIMEOUT", 5: "PTCA_ERR_NUMERIC", 6: "PTCA_ERR_UNSUPPORTED"}
SCHEDULE_TILED, SCHEDULE_BLOCK = 0, 1
PIPELINE_STAGES, PIPELINE_PERSISTENT, PIPELINE_GRAPH, PIPELINE_OVERLAP = 0, 1, 2, 3
REDUCTION_ROWS, REDUCTION_TILED, REDUCTION_SHARED = 0, 1, 2
FP64, MIXED = 0, 1
PROPOSAL_SPHERE, PROPOSAL_CONE = 0, 1
MODEL_DOUBLE_EXCHANGE, MODEL_HUBBARD_MF, MODEL_HOLSTEIN = 0, 1, 2

EXPORTED = [
    "ptca_init", "ptca_destroy", "ptca_set_T", "ptca_set_mu", "ptca_get_spins", "ptca_set_spins",
    "ptca_dims", "ptca_build_clusters", "ptca_cluster_eigvals", "ptca_free_energy", "ptca_sweep",
    "ptca_sweep_record", "ptca_observables", "ptca_schedule", "ptca_last_error", "ptca_version",
    "ptca_sweep_noalloc", "ptca_set_pipeline", "ptca_selftest_barrier_timeout", "ptca_set_resolve_margin",
    "ptca_surrogate_param_count", "ptca_surrogate_init", "ptca_surrogate_get_params", "ptca_surrogate_set_params",
    "ptca_surrogate_collect", "ptca_surrogate_train", "ptca_surrogate_grad", "ptca_surrogate_predict",
    "ptca_surrogate_enable", "ptca_set_checker", "ptca_checker_read", "ptca_set_launch_config",
    "ptca_get_launch_config", "ptca_autotune", "ptca_set_kernel_timing", "ptca_kernel_times",
    "ptca_stage_split", "ptca_full_spectrum", "ptca_stage_run", "ptca_get_sites", "ptca_set_sites", "ptca_flush",
]


class PtcaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class LaunchConfig(ctypes.Structure):
    _fields_ = [("pipeline", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("reduction", ctypes.c_int32), ("panel_width", ctypes.c_int32)]


class Lattice(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32), ("periodic", ctypes.c_int32), ("Lz", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double), ("J_H", ctypes.c_double), ("mu", ctypes.c_double), ("T", ctypes.c_double),
        ("L_c", ctypes.c_int32), ("cluster_periodic", ctypes.c_int32), ("update_offset", ctypes.c_int32),
        ("schedule", ctypes.c_int32), ("stride", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("proposal", ctypes.c_int32), ("model", ctypes.c_int32), ("cone_deg", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("U", ctypes.c_double), ("m_step", ctypes.c_double),
        ("lam", ctypes.c_double), ("K", ctypes.c_double),
    ]


class SweepStats(ctypes.Structure):
    _fields_ = [("attempts", ctypes.c_int64), ("accepted", ctypes.c_int64), ("eigensolves", ctypes.c_int64),
                ("resolved", ctypes.c_int64), ("sweeps", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("screened", ctypes.c_int64)]


class Obs(ctypes.Structure):
    _fields_ = [("S_00", ctypes.c_double), ("S_pipi", ctypes.c_double), ("F_site", ctypes.c_double),
                ("acceptance", ctypes.c_double), ("filling", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libptca.so (it must have been built; see ``__graft_entry__.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        P = ctypes.POINTER
        sig = {
            "ptca_init": ([P(Lattice), P(Params), P(vp)], i32),
            "ptca_destroy": ([vp], i32),
            "ptca_set_T": ([vp, dbl], i32),
            "ptca_set_mu": ([vp, dbl], i32),
            "ptca_get_spins": ([vp, vp, ctypes.c_int, vp], i32),
            "ptca_set_spins": ([vp, vp, ctypes.c_int, vp], i32),
            "ptca_dims": ([vp, P(i32), P(i64)], i32),
            "ptca_build_clusters": ([vp, vp, i32, vp, vp, vp, vp, vp], i32),
            "ptca_cluster_eigvals": ([vp, vp, vp, vp, i32, vp, vp, vp], i32),
            "ptca_free_energy": ([vp, vp, vp, vp, i32, dbl, dbl, vp, vp], i32),
            "ptca_sweep": ([vp, i32, P(SweepStats), vp], i32),
            "ptca_sweep_record": ([vp, vp, vp, vp, vp, vp, vp], i32),
            "ptca_observables": ([vp, P(Obs), vp], i32),
            "ptca_schedule": ([P(Lattice), P(Params), vp, vp, P(i32)], i32),
            "ptca_stage_split": ([P(Lattice), P(Params), vp, vp], i32),
            "ptca_full_spectrum": ([vp, vp, vp], i32),
            "ptca_last_error": ([], ctypes.c_char_p),
            "ptca_version": ([], i32),
            "ptca_sweep_noalloc": ([P(Lattice), P(Params), vp, i64, vp, vp, vp, vp], i32),
            "ptca_set_pipeline": ([vp, i32, dbl], i32),
            "ptca_set_resolve_margin": ([vp, dbl], i32),
            "ptca_set_checker": ([vp, i32], i32),
            "ptca_set_launch_config": ([vp, P(LaunchConfig)], i32),
            "ptca_get_launch_config": ([vp, P(LaunchConfig)], i32),
            "ptca_autotune": ([vp, i32, P(LaunchConfig), ctypes.c_char_p, i32, vp], i32),
            "ptca_set_kernel_timing": ([vp, i32], i32),
            "ptca_kernel_times": ([vp, vp, vp], i32),
            "ptca_checker_read": ([vp, vp, i32, vp], i32),
            "ptca_surrogate_param_count": ([], i32),
            "ptca_surrogate_init": ([vp, ctypes.c_uint64, vp], i32),
            "ptca_surrogate_get_params": ([vp, vp, P(ctypes.c_float), vp], i32),
            "ptca_surrogate_set_params": ([vp, vp, ctypes.c_float, vp], i32),
            "ptca_surrogate_collect": ([vp, i32, vp, vp, vp, vp], i32),
            "ptca_surrogate_train": ([vp, vp, vp, vp, i64, i32, i32, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_uint64, vp, vp], i32),
            "ptca_surrogate_grad": ([vp, vp, vp, vp, i32, vp, vp, vp], i32),
            "ptca_surrogate_predict": ([vp, vp, vp, i32, vp, vp], i32),
            "ptca_surrogate_enable": ([vp, i32], i32),
            "ptca_selftest_barrier_timeout": ([i32, dbl, vp], i32),
            "ptca_stage_run": ([vp, i64, vp, i32, vp], i32),
            "ptca_flush": ([vp, vp], i32),
            "ptca_get_sites": ([vp, vp, i32, vp, i32, vp], i32),
            "ptca_set_sites": ([vp, vp, i32, vp, i32, vp], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def _check(status: int):
    if status != PTCA_OK:
        raise PtcaError(status, lib().ptca_last_error().decode())


def _ptr(t):
    """Raw pointer of a tensor / numpy array / None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    if hasattr(t, "ctypes"):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(int(t))


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


@dataclass
class Config:
    """Problem definition, mirrored into ptca_lattice / ptca_params."""
    Lx: int
    Ly: int
    L_c: int
    periodic: int = 1
    t: float = 1.0
    J_H: float = 8.0
    mu: float = -6.5
    T: float = 0.05
    cluster_periodic: int = -1
    update_offset: int = -1
    schedule: int = SCHEDULE_TILED
    stride: int = 0
    precision: int = FP64
    proposal: int = PROPOSAL_SPHERE
    cone_deg: float = 30.0
    seed: int = 0
    model: int = MODEL_DOUBLE_EXCHANGE
    U: float = 8.0
    m_step: float = 0.5
    Lz: int = 1
    lam: float = 1.0
    K: float = 1.0

    def lattice(self) -> Lattice:
        return Lattice(self.Lx, self.Ly, self.periodic, self.Lz)

    def params(self) -> Params:
        return Params(self.t, self.J_H, self.mu, self.T, self.L_c, self.cluster_periodic, self.update_offset,
                      self.schedule, self.stride, self.precision, self.proposal, self.model, self.cone_deg,
                      self.seed, self.U, self.m_step, self.lam, self.K)

    @property
    def N(self) -> int:
        return self.Lx * self.Ly * self.Lz


# ---------------------------------------------------------------------------
# Functions with the C names (pointer/size marshalling only)
# ---------------------------------------------------------------------------
def ptca_version() -> int:
    return lib().ptca_version()


def ptca_last_error() -> str:
    """Description of the last failure on this thread."""
    return lib().ptca_last_error().decode()


def ptca_schedule(cfg: Config):
    """Host-only schedule: list of int32 numpy arrays (one per stage)."""
    import numpy as np
    N = cfg.N
    start = np.zeros(N + 1, dtype=np.int32)
    sites = np.zeros(N, dtype=np.int32)
    ns = ctypes.c_int32()
    lat, par = cfg.lattice(), cfg.params()
    _check(lib().ptca_schedule(ctypes.byref(lat), ctypes.byref(par), _ptr(start), _ptr(sites), ctypes.byref(ns)))
    return [sites[start[s]:start[s + 1]].copy() for s in range(ns.value)]


def ptca_stage_split(cfg: Config):
    """Host-only dependence split of every stage on the stage before it: list
    of (order, n_indep) per stage, order = int32 indices into the stage's site
    list, the n_indep visits whose windows hold no site of the previous stage
    first."""
    import numpy as np
    stages = ptca_schedule(cfg)
    order = np.zeros(cfg.N, dtype=np.int32)
    indep = np.zeros(len(stages), dtype=np.int32)
    lat, par = cfg.lattice(), cfg.params()
    _check(lib().ptca_stage_split(ctypes.byref(lat), ctypes.byref(par), _ptr(order), _ptr(indep)))
    out, o = [], 0
    for s, sites in enumerate(stages):
        out.append((order[o:o + sites.size].copy(), int(indep[s])))
        o += sites.size
    return out


def ptca_init(cfg: Config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    lat, par = cfg.lattice(), cfg.params()
    _check(lib().ptca_init(ctypes.byref(lat), ctypes.byref(par), ctypes.byref(h)))
    return h


def ptca_destroy(h) -> None:
    _check(lib().ptca_destroy(h))


def ptca_set_T(h, T: float) -> None:
    _check(lib().ptca_set_T(h, T))


def ptca_set_mu(h, mu: float) -> None:
    _check(lib().ptca_set_mu(h, mu))


def ptca_get_spins(h, dst, stream=None) -> None:
    on_dev = int(getattr(dst, "is_cuda", False))
    _check(lib().ptca_get_spins(h, _ptr(dst), on_dev, _stream(stream)))


def ptca_set_spins(h, src, stream=None) -> None:
    on_dev = int(getattr(src, "is_cuda", False))
    _check(lib().ptca_set_spins(h, _ptr(src), on_dev, _stream(stream)))


def ptca_dims(h):
    nmax, stride = ctypes.c_int32(), ctypes.c_int64()
    _check(lib().ptca_dims(h, ctypes.byref(nmax), ctypes.byref(stride)))
    return nmax.value, stride.value


def ptca_build_clusters(h, sites, m, new_spins, H_out, offsets_out, n_out, stream=None) -> None:
    _check(lib().ptca_build_clusters(h, _ptr(sites), m, _ptr(new_spins), _ptr(H_out), _ptr(offsets_out),
                                     _ptr(n_out), _stream(stream)))


def ptca_cluster_eigvals(h, H, offsets, n, m, eig_out, eig_offsets, stream=None) -> None:
    _check(lib().ptca_cluster_eigvals(h, _ptr(H), _ptr(offsets), _ptr(n), m, _ptr(eig_out), _ptr(eig_offsets),
                                      _stream(stream)))


def ptca_free_energy(h, eig, eig_offsets, n, m, mu, T, F_out, stream=None) -> None:
    _check(lib().ptca_free_energy(h, _ptr(eig), _ptr(eig_offsets), _ptr(n), m, mu, T, _ptr(F_out),
                                  _stream(stream)))


def ptca_sweep(h, n_sweeps: int, stats: bool = True, stream=None):
    st = SweepStats() if stats else None
    _check(lib().ptca_sweep(h, n_sweeps, ctypes.byref(st) if stats else None, _stream(stream)))
    return st


def ptca_sweep_record(h, site=None, F_old=None, F_new=None, lnu=None, accepted=None, stream=None) -> None:
    _check(lib().ptca_sweep_record(h, _ptr(site), _ptr(F_old), _ptr(F_new), _ptr(lnu), _ptr(accepted),
                                   _stream(stream)))


def ptca_sweep_noalloc(cfg: Config, spins, sweep_index: int, F_out=None, accepted_out=None, status_out=None,
                       stream=None) -> None:
    """One sweep without a context or device allocation (see include/ptca.h).

    spins: CUDA float64 tensor (N, 3), updated in place; F_out: CUDA float64
    (2N,) or None; accepted_out: CUDA uint8 (N,) or None, in the flattened
    order of ptca_schedule(cfg); status_out: CUDA int32 (1,) or None."""
    import torch
    N = cfg.N

    def need(t, name, dtype, numel):
        if t is None:
            return
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
            raise ValueError(f"{name} must be a contiguous {dtype} tensor of {numel} elements")

    if spins is None:
        raise ValueError("spins is required")
    need(spins, "spins", torch.float64, 3 * N)
    need(F_out, "F_out", torch.float64, 2 * N)
    need(accepted_out, "accepted_out", torch.uint8, N)
    need(status_out, "status_out", torch.int32, 1)
    lat, par = cfg.lattice(), cfg.params()
    _check(lib().ptca_sweep_noalloc(ctypes.byref(lat), ctypes.byref(par), _ptr(spins), sweep_index, _ptr(F_out),
                                    _ptr(accepted_out), _ptr(status_out), _stream(stream)))


def ptca_flush(h, stream=None) -> None:
    """Complete, stream-ordered, a re-solve the last overlapped sweep left running."""
    _check(lib().ptca_flush(h, _stream(stream)))


def ptca_stage_run(h, sweep_index: int, sites, stream=None) -> None:
    """The given visits (host int32 site list, one stage) of sweep `sweep_index`."""
    import numpy as np
    s = np.ascontiguousarray(sites, dtype=np.int32)
    _check(lib().ptca_stage_run(h, sweep_index, _ptr(s), s.size, _stream(stream)))


def ptca_get_sites(h, sites, out, stream=None) -> None:
    """Spins of the listed sites (host int32 list) into `out` (float64, 3 per
    site; a CUDA tensor stays stream-ordered, a host array synchronises)."""
    import numpy as np
    s = np.ascontiguousarray(sites, dtype=np.int32)
    _check(lib().ptca_get_sites(h, _ptr(s), s.size, _ptr(out), int(getattr(out, 'is_cuda', False)), _stream(stream)))


def ptca_set_sites(h, sites, spins, stream=None) -> None:
    """Write the spins (float64, 3 per listed site) of the listed sites."""
    import numpy as np
    s = np.ascontiguousarray(sites, dtype=np.int32)
    _check(lib().ptca_set_sites(h, _ptr(s), s.size, _ptr(spins), int(getattr(spins, 'is_cuda', False)), _stream(stream)))


def ptca_set_pipeline(h, mode: int, barrier_timeout_s: float = 30.0) -> None:
    _check(lib().ptca_set_pipeline(h, mode, barrier_timeout_s))


def ptca_set_resolve_margin(h, margin: float) -> None:
    _check(lib().ptca_set_resolve_margin(h, margin))


def ptca_set_launch_config(h, pipeline: int, warps_per_cta: int = 8, ctas_per_sm: int = 0, reduction: int = 0,
                           panel_width: int = 0) -> None:
    _check(lib().ptca_set_launch_config(h, ctypes.byref(LaunchConfig(pipeline, warps_per_cta, ctas_per_sm, reduction,
                                                                     panel_width))))


def ptca_get_launch_config(h) -> LaunchConfig:
    out = LaunchConfig()
    _check(lib().ptca_get_launch_config(h, ctypes.byref(out)))
    return out


def ptca_autotune(h, trial_sweeps: int = 3, stream=None):
    """Time every launch configuration, apply the fastest; returns (best, table)
    with table the parsed JSON of every candidate."""
    import json
    best = LaunchConfig()
    buf = ctypes.create_string_buffer(1 << 14)
    _check(lib().ptca_autotune(h, trial_sweeps, ctypes.byref(best), buf, len(buf), _stream(stream)))
    return best, json.loads(buf.value.decode())


def ptca_set_kernel_timing(h, on: bool) -> None:
    _check(lib().ptca_set_kernel_timing(h, 1 if on else 0))


# Per-kernel CUDA-event totals since the last read (see ptca_kernel_times).
KernelTimes = namedtuple("KernelTimes", ["stage_ms", "stage_launches", "resolve_ms", "resolve_launches",
                                         "dependent_ms", "dependent_launches", "stage_matrices",
                                         "dependent_matrices", "stage_union_ms"])


def ptca_kernel_times(h, stream=None) -> KernelTimes:
    """(stage_ms, stage_launches, resolve_ms, resolve_launches, dependent_ms,
    dependent_launches, stage_matrices, dependent_matrices) since the last
    call; clears the record.  The dependent_* entries are the overlapped
    pipeline's launches of the visits that wait for the previous stage's
    re-solve; stage_* are all other stage launches; stage_union_ms is the
    time at least one stage launch ran (look-ahead launches overlap)."""
    import numpy as np
    out = np.zeros(9, dtype=np.float64)
    _check(lib().ptca_kernel_times(h, _ptr(out), _stream(stream)))
    return KernelTimes(float(out[0]), int(out[1]), float(out[2]), int(out[3]), float(out[4]), int(out[5]),
                       int(out[6]), int(out[7]), float(out[8]))


def ptca_full_spectrum(h, eig_out, stream=None) -> None:
    """All 2N eigenvalues of the whole lattice's one-body Hamiltonian (device
    float64 tensor of 2N entries, filled ascending)."""
    _check(lib().ptca_full_spectrum(h, _ptr(eig_out), _stream(stream)))


def ptca_set_checker(h, on: bool) -> None:
    _check(lib().ptca_set_checker(h, 1 if on else 0))


def ptca_checker_read(h, n_stages: int, stream=None):
    """Per-stage precision-checker maxima since the last read: numpy array
    (n_stages, 5) = |d eps|, |d dF|, |d eps|/(J_H+4|t|), |d dF|/max(1,|F|),
    |d dF| / max(|dF|, sum_k |eps_k-mu| f_k / n)."""
    import numpy as np
    out = np.zeros((n_stages, 5), dtype=np.float64)
    _check(lib().ptca_checker_read(h, _ptr(out), n_stages, _stream(stream)))
    return out


def ptca_surrogate_param_count() -> int:
    return lib().ptca_surrogate_param_count()


def ptca_surrogate_init(h, seed: int = 0, stream=None) -> None:
    _check(lib().ptca_surrogate_init(h, seed, _stream(stream)))


def ptca_surrogate_get_params(h, theta, stream=None) -> float:
    sc = ctypes.c_float()
    _check(lib().ptca_surrogate_get_params(h, _ptr(theta), ctypes.byref(sc), _stream(stream)))
    return sc.value


def ptca_surrogate_set_params(h, theta, scale: float, stream=None) -> None:
    _check(lib().ptca_surrogate_set_params(h, _ptr(theta), scale, _stream(stream)))


def ptca_surrogate_collect(h, n_sweeps: int, feat, center, dF, stream=None) -> None:
    _check(lib().ptca_surrogate_collect(h, n_sweeps, _ptr(feat), _ptr(center), _ptr(dF), _stream(stream)))


def ptca_surrogate_train(h, feat, center, dF, n: int, steps: int, batch: int, lr: float, weight_decay: float,
                         seed: int, loss_trace=None, stream=None) -> None:
    _check(lib().ptca_surrogate_train(h, _ptr(feat), _ptr(center), _ptr(dF), n, steps, batch, lr, weight_decay, seed,
                                      _ptr(loss_trace), _stream(stream)))


def ptca_surrogate_grad(h, feat, center, dF, n: int, grad_out, loss_out, stream=None) -> None:
    _check(lib().ptca_surrogate_grad(h, _ptr(feat), _ptr(center), _ptr(dF), n, _ptr(grad_out), _ptr(loss_out),
                                     _stream(stream)))


def ptca_surrogate_predict(h, feat, center, n: int, dF_out, stream=None) -> None:
    _check(lib().ptca_surrogate_predict(h, _ptr(feat), _ptr(center), n, _ptr(dF_out), _stream(stream)))


def ptca_surrogate_enable(h, on: bool) -> None:
    _check(lib().ptca_surrogate_enable(h, int(bool(on))))


def ptca_selftest_barrier_timeout(blocks: int, timeout_s: float, stream=None) -> int:
    """Returns the raw status (PTCA_ERR_TIMEOUT = 4 is the expected outcome)."""
    st = lib().ptca_selftest_barrier_timeout(blocks, timeout_s, _stream(stream))
    return st


def ptca_observables(h, stream=None) -> Obs:
    o = Obs()
    _check(lib().ptca_observables(h, ctypes.byref(o), _stream(stream)))
    return o


# ---------------------------------------------------------------------------
# Convenience wrapper owning a context
# ---------------------------------------------------------------------------
class Context:
    """A PTCA problem on the current CUDA device.

    Uses torch only to allocate device buffers for the batched calls.
    """

    def __init__(self, cfg: Config):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA GPU is required (no CPU fallback)")
        self.cfg = cfg
        self.h = ptca_init(cfg)
        self.nmax, self.packed_stride = ptca_dims(self.h)

    def close(self):
        if self.h:
            ptca_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def N(self):
        return self.cfg.N

    def spins(self):
        import torch
        out = torch.empty((self.N, 3), dtype=torch.float64, device="cuda")
        ptca_get_spins(self.h, out)
        return out

    def set_spins(self, S):
        import torch
        S = torch.as_tensor(S, dtype=torch.float64).contiguous()
        if not S.is_cuda:
            S = S.cuda()
        ptca_set_spins(self.h, S)

    def sweep(self, n: int = 1, stats: bool = True):
        return ptca_sweep(self.h, n, stats)

    def record(self):
        import torch
        N = self.N
        site = torch.empty(N, dtype=torch.int32, device="cuda")
        Fo = torch.empty(N, dtype=torch.float64, device="cuda")
        Fn = torch.empty(N, dtype=torch.float64, device="cuda")
        lnu = torch.empty(N, dtype=torch.float64, device="cuda")
        acc = torch.empty(N, dtype=torch.uint8, device="cuda")
        ptca_sweep_record(self.h, site, Fo, Fn, lnu, acc)
        torch.cuda.synchronize()
        return site, Fo, Fn, lnu, acc

    def observables(self) -> Obs:
        return ptca_observables(self.h)

    def build_clusters(self, sites, new_spins=None):
        """Packed cluster matrices for update sites (device tensors)."""
        import torch
        sites = torch.as_tensor(sites, dtype=torch.int32).cuda().contiguous()
        m = sites.numel()
        dt = torch.complex128 if self.cfg.precision == FP64 else torch.complex64
        H = torch.zeros(max(m, 1) * self.packed_stride, dtype=dt, device="cuda")
        offs = torch.zeros(max(m, 1), dtype=torch.int64, device="cuda")
        n = torch.zeros(max(m, 1), dtype=torch.int32, device="cuda")
        ns = None
        if new_spins is not None:
            ns = torch.as_tensor(new_spins, dtype=torch.float64).cuda().contiguous()
        ptca_build_clusters(self.h, sites, m, ns, H, offs, n)
        return H, offs[:m], n[:m]

    def cluster_eigvals(self, H, offsets, n):
        import torch
        m = n.numel()
        eoff = torch.arange(m, dtype=torch.int64, device="cuda") * self.nmax
        eig = torch.full((max(m, 1) * self.nmax,), float("nan"), dtype=torch.float64, device="cuda")
        ptca_cluster_eigvals(self.h, H, offsets, n, m, eig, eoff)
        return eig[: m * self.nmax].view(m, self.nmax) if m else eig[:0].view(0, self.nmax), eoff

    def free_energy(self, eig_flat, eoff, n, mu=None, T=None):
        import torch
        m = n.numel()
        F = torch.empty(max(m, 1), dtype=torch.float64, device="cuda")
        ptca_free_energy(self.h, eig_flat, eoff, n, m, self.cfg.mu if mu is None else mu,
                         self.cfg.T if T is None else T, F)
        return F[:m]
