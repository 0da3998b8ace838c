"""Plain FP64 CPU oracle for the traveling-cluster Monte Carlo hot path.

TEST INFRASTRUCTURE ONLY.  The product library never imports this package.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  The arithmetic lives in ``ptca_oracle.c`` (plain C,
FP64, no fast-math, no FMA contraction); this module compiles it with gcc and
exposes it through ctypes with numpy arrays.

What each function follows (paper sections):
  * ``cluster_hamiltonian`` -- the cluster Hamiltonian H_clus{C[i_s]} built
    around an update site (Sec. II.b-c, Fig. 1), periodic on the cluster
    (Sec. II.b), two spin species per site (Sec. IV, 2N x 2N matrices); the
    model is the double-exchange Hamiltonian (-t hopping, -J_H S.sigma) or the
    Hubbard mean-field Hamiltonian of Eq. 1 with <n_i> = 1 (on-site
    (U/2)(n_i - m_i.sigma), classical energy (U/4)(m_i^2 - 1) per window site
    in the cluster free energy), chosen by ``Model.model``.
  * ``eigvalsh`` -- cyclic complex Jacobi diagonalisation (Sec. II.c step b).
  * ``free_energy`` -- grand-canonical one-body free energy of the cluster
    (Sec. II.b: the periodic cluster is a grand-canonical ensemble).
  * ``sweep`` -- one sequential TCA sweep, steps a-f of Sec. II.c, visiting
    the sites in the flattened order of a PTCA schedule (Sec. III.a).
  * ``schedule`` -- the stage lists of Sec. III.a (2^d blocks) and a tiled
    sublattice schedule.
  * ``structure_factor`` -- Eq. 2 for one configuration.
"""
from __future__ import annotations

import ctypes
import fcntl
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ptca_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libptca_oracle.so")
_SAN_PATH = os.path.join(_BUILD, "libptca_oracle_san.so")
_lock = threading.Lock()
_lib = None

SCHEDULE_TILED = 0
SCHEDULE_BLOCK = 1
MODEL_DOUBLE_EXCHANGE = 0
MODEL_HUBBARD_MF = 1
MODEL_HOLSTEIN = 2
PROPOSAL_SPHERE = 0
PROPOSAL_CONE = 1


def build(force: bool = False, sanitize: bool = False) -> str:
    """Compile the C oracle with gcc (no fast-math, no FMA contraction).
    With sanitize, a separate copy instrumented by AddressSanitizer and
    UndefinedBehaviorSanitizer, every finding fatal; it loads only into a
    process that has the ASan runtime preloaded."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _SAN_PATH if sanitize else _LIB_PATH

    def fresh():
        return os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC)

    if not force and fresh():
        return path
    with open(os.path.join(_BUILD, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)  # one builder at a time
        if not force and fresh():
            return path
        tmp = path + f".{os.getpid()}.tmp"
        extra = (["-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined", "-fno-sanitize-recover=all"]
                 if sanitize else [])
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", *extra, "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
    return path


class _Model(ctypes.Structure):
    _fields_ = [
        ("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32),
        ("lattice_periodic", ctypes.c_int32), ("Lc", ctypes.c_int32),
        ("ox", ctypes.c_int32), ("oy", ctypes.c_int32),
        ("cluster_periodic", ctypes.c_int32), ("schedule", ctypes.c_int32),
        ("stride", ctypes.c_int32), ("proposal", ctypes.c_int32),
        ("t", ctypes.c_double), ("JH", ctypes.c_double),
        ("mu", ctypes.c_double), ("T", ctypes.c_double),
        ("cone_deg", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("model", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("U", ctypes.c_double), ("m_step", ctypes.c_double),
        ("Lz", ctypes.c_int32), ("oz", ctypes.c_int32),
        ("lam", ctypes.c_double), ("K", ctypes.c_double),
    ]


@dataclass
class Model:
    """One oracle problem.  ``ox``/``oy`` default to the schedule's update-site
    offset: floor(L_c/2) for the tiled schedule (central site), 0 for the
    block schedule (corner site, Sec. III.a)."""
    Lx: int
    Ly: int
    Lc: int
    t: float = 1.0
    JH: float = 8.0
    mu: float = -6.5
    T: float = 0.05
    lattice_periodic: int = 1
    cluster_periodic: int = -1
    schedule: int = SCHEDULE_TILED
    stride: int = 0
    proposal: int = PROPOSAL_SPHERE
    cone_deg: float = 30.0
    seed: int = 0
    ox: int = -1
    oy: int = -1
    model: int = MODEL_DOUBLE_EXCHANGE
    U: float = 8.0
    m_step: float = 0.5
    Lz: int = 1
    oz: int = -1
    lam: float = 1.0
    K: float = 1.0

    def _c(self) -> _Model:
        off = (self.Lc // 2) if self.schedule == SCHEDULE_TILED else 0
        ox = off if self.ox < 0 else self.ox
        oy = (off if self.oy < 0 else self.oy) if self.Ly > 1 else 0
        oz = (off if self.oz < 0 else self.oz) if self.Lz > 1 else 0
        cp = self.lattice_periodic if self.cluster_periodic < 0 else self.cluster_periodic
        stride = self.stride if self.stride > 0 else self.Lc
        return _Model(self.Lx, self.Ly, self.lattice_periodic, self.Lc, ox, oy, cp,
                      self.schedule, stride, self.proposal, self.t, self.JH,
                      self.mu, self.T, self.cone_deg, self.seed, self.model, 0, self.U, self.m_step,
                      self.Lz, oz, self.lam, self.K)

    @property
    def N(self) -> int:
        return self.Lx * self.Ly * self.Lz

    @property
    def nmax(self) -> int:
        return 2 * self.Lc ** (1 + (self.Ly > 1) + (self.Lz > 1))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # PTCA_ORACLE_LIB selects another build of the same source (the
            # sanitizer-instrumented copy).
            _lib = ctypes.CDLL(os.environ.get("PTCA_ORACLE_LIB") or build())
            P = ctypes.POINTER
            d, i32, u32, u64, u8 = (ctypes.c_double, ctypes.c_int32, ctypes.c_uint32,
                                    ctypes.c_uint64, ctypes.c_uint8)
            M = P(_Model)
            _lib.oracle_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
            _lib.oracle_uniform2.argtypes = [u64, u64, u32, u32, P(d)]
            _lib.oracle_init_spins.argtypes = [M, P(d)]
            _lib.oracle_propose.argtypes = [M, u64, ctypes.c_int, P(d), P(d)]
            _lib.oracle_cluster_hamiltonian.argtypes = [M, P(d), ctypes.c_int, P(d), P(d),
                                                        P(ctypes.c_int), P(ctypes.c_int)]
            _lib.oracle_cluster_hamiltonian.restype = ctypes.c_int
            _lib.oracle_eigvalsh_jacobi.argtypes = [ctypes.c_int, P(d), P(d)]
            _lib.oracle_eigvalsh_jacobi.restype = ctypes.c_int
            _lib.oracle_free_energy.argtypes = [ctypes.c_int, P(d), d, d]
            _lib.oracle_free_energy.restype = d
            _lib.oracle_schedule.argtypes = [M, P(i32), P(i32)]
            _lib.oracle_schedule.restype = ctypes.c_int
            _lib.oracle_in_window.argtypes = [M, ctypes.c_int, ctypes.c_int]
            _lib.oracle_in_window.restype = ctypes.c_int
            _lib.oracle_sweep.argtypes = [M, P(d), u64, P(i32), P(d), P(d), P(d), P(u8)]
            _lib.oracle_sweep.restype = ctypes.c_int
            _lib.oracle_single_site_chain.argtypes = [M, P(d), ctypes.c_int, u64, ctypes.c_int, P(d)]
            _lib.oracle_single_site_chain.restype = ctypes.c_int
            _lib.oracle_cluster_free_energy.argtypes = [M, P(d), ctypes.c_int, P(d)]
            _lib.oracle_cluster_free_energy.restype = d
            _lib.oracle_structure_factor.argtypes = [ctypes.c_int, ctypes.c_int, P(d), d, d]
            _lib.oracle_structure_factor.restype = d
            _lib.oracle_structure_factor3.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P(d), d, d, d]
            _lib.oracle_structure_factor3.restype = d
        return _lib


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(key, ctr) -> np.ndarray:
    k = np.ascontiguousarray(key, dtype=np.uint32)
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(k, ctypes.c_uint32), _p(c, ctypes.c_uint32),
                               _p(out, ctypes.c_uint32))
    return out


def uniform2(seed: int, sweep: int, site: int, purpose: int) -> np.ndarray:
    u = np.zeros(2)
    lib().oracle_uniform2(seed, sweep, site, purpose, _p(u, ctypes.c_double))
    return u


def init_spins(m: Model) -> np.ndarray:
    S = np.zeros((m.N, 3))
    cm = m._c()
    lib().oracle_init_spins(ctypes.byref(cm), _p(S, ctypes.c_double))
    return S


def propose(m: Model, sweep: int, site: int, s_old) -> np.ndarray:
    so = np.ascontiguousarray(s_old, dtype=np.float64)
    sn = np.zeros(3)
    cm = m._c()
    lib().oracle_propose(ctypes.byref(cm), sweep, site, _p(so, ctypes.c_double),
                         _p(sn, ctypes.c_double))
    return sn


def cluster_hamiltonian(m: Model, S, site: int, s_new=None):
    """Dense n x n complex cluster matrix, plus the window extents (ex, ey)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    H = np.zeros((m.nmax, m.nmax), dtype=np.complex128)
    ex, ey = ctypes.c_int(), ctypes.c_int()
    sn = None if s_new is None else np.ascontiguousarray(s_new, dtype=np.float64)
    cm = m._c()
    n = lib().oracle_cluster_hamiltonian(
        ctypes.byref(cm), _p(S, ctypes.c_double), site,
        None if sn is None else _p(sn, ctypes.c_double),
        H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(ex), ctypes.byref(ey))
    Hn = H.reshape(-1)[: n * n].reshape(n, n).copy()
    return Hn, (ex.value, ey.value)


def eigvalsh(H) -> np.ndarray:
    """Eigenvalues (ascending) of a complex Hermitian matrix by cyclic Jacobi."""
    A = np.array(H, dtype=np.complex128, order="C", copy=True)
    n = A.shape[0]
    e = np.zeros(n)
    sweeps = lib().oracle_eigvalsh_jacobi(n, A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          _p(e, ctypes.c_double))
    if sweeps < 0:
        raise RuntimeError("Jacobi did not converge in 100 sweeps")
    return e


def free_energy(eig, mu: float, T: float) -> float:
    e = np.ascontiguousarray(eig, dtype=np.float64)
    return lib().oracle_free_energy(e.size, _p(e, ctypes.c_double), mu, T)


def cluster_free_energy(m: Model, S, site: int, s_new=None) -> float:
    S = np.ascontiguousarray(S, dtype=np.float64)
    sn = None if s_new is None else np.ascontiguousarray(s_new, dtype=np.float64)
    cm = m._c()
    return lib().oracle_cluster_free_energy(ctypes.byref(cm), _p(S, ctypes.c_double), site,
                                            None if sn is None else _p(sn, ctypes.c_double))


def schedule(m: Model):
    """List of stages, each an int32 array of update sites."""
    N = m.N
    starts = np.zeros(N + 1, dtype=np.int32)
    sites = np.zeros(N, dtype=np.int32)
    cm = m._c()
    ns = lib().oracle_schedule(ctypes.byref(cm), _p(starts, ctypes.c_int32),
                               _p(sites, ctypes.c_int32))
    return [sites[starts[s]:starts[s + 1]].copy() for s in range(ns)]


def in_window(m: Model, centre: int, site: int) -> bool:
    cm = m._c()
    return bool(lib().oracle_in_window(ctypes.byref(cm), centre, site))


@dataclass
class SweepRecord:
    site: np.ndarray
    F_old: np.ndarray
    F_new: np.ndarray
    lnu: np.ndarray
    accepted: np.ndarray


def sweep(m: Model, S, sweep_index: int):
    """One sequential TCA sweep; returns (new spins, per-visit record)."""
    S = np.array(S, dtype=np.float64, order="C", copy=True)
    N = m.N
    rec = SweepRecord(np.zeros(N, np.int32), np.zeros(N), np.zeros(N), np.zeros(N),
                      np.zeros(N, np.uint8))
    cm = m._c()
    nacc = lib().oracle_sweep(ctypes.byref(cm), _p(S, ctypes.c_double), sweep_index,
                              _p(rec.site, ctypes.c_int32), _p(rec.F_old, ctypes.c_double),
                              _p(rec.F_new, ctypes.c_double), _p(rec.lnu, ctypes.c_double),
                              _p(rec.accepted, ctypes.c_uint8))
    if nacc < 0:
        raise MemoryError("oracle sweep allocation failed")
    return S, rec


def single_site_chain(m: Model, S, site: int, sweep0: int, steps: int):
    S = np.array(S, dtype=np.float64, order="C", copy=True)
    trace = np.zeros((steps, 3))
    cm = m._c()
    nacc = lib().oracle_single_site_chain(ctypes.byref(cm), _p(S, ctypes.c_double), site,
                                          sweep0, steps, _p(trace, ctypes.c_double))
    return trace, nacc


def structure_factor(Lx: int, Ly: int, S, qx: float, qy: float, Lz: int = 1, qz: float = 0.0) -> float:
    S = np.ascontiguousarray(S, dtype=np.float64)
    return lib().oracle_structure_factor3(Lx, Ly, Lz, _p(S, ctypes.c_double), qx, qy, qz)
