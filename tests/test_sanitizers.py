"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer (no GPU).

- The C oracle: it is the reference every GPU result is checked against, so an
  out-of-bounds read or an undefined operation in it would silently corrupt
  the expected values.  Every entry point runs: each model, chains, square and
  cubic lattices, open and periodic, both schedules, both proposals.
- The host side of the C ABI: validation, schedules and their exactness
  check, the stage split, error reporting.

Each runs in a child process with the ASan runtime preloaded and every
finding fatal.
"""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

EXERCISE = r"""
import numpy as np
import oracle
from tests import inputs

cases = [
    oracle.Model(Lx=8, Ly=8, Lc=4, T=0.05, seed=0),
    oracle.Model(Lx=8, Ly=8, Lc=4, schedule=oracle.SCHEDULE_BLOCK, proposal=oracle.PROPOSAL_CONE, seed=1),
    oracle.Model(Lx=7, Ly=5, Lc=4, lattice_periodic=0, stride=4, JH=6.0, mu=-4.5, T=0.1, seed=2),
    oracle.Model(Lx=8, Ly=1, Lc=4, schedule=oracle.SCHEDULE_BLOCK, JH=4.0, mu=-3.0, T=0.2, seed=3),
    oracle.Model(Lx=6, Ly=6, Lc=2, model=oracle.MODEL_HUBBARD_MF, U=8.0, mu=4.0, T=0.1, seed=4),
    oracle.Model(Lx=16, Ly=1, Lc=4, model=oracle.MODEL_HOLSTEIN, lam=1.5, K=1.0, mu=0.0, T=0.1,
                 schedule=oracle.SCHEDULE_BLOCK, seed=5),
    oracle.Model(Lx=4, Ly=4, Lz=4, Lc=2, schedule=oracle.SCHEDULE_BLOCK, JH=6.0, seed=6),
    oracle.Model(Lx=5, Ly=4, Lz=3, Lc=3, lattice_periodic=0, schedule=oracle.SCHEDULE_BLOCK, seed=7),
]
for m in cases:
    N = m.Lx * m.Ly * m.Lz
    S = oracle.init_spins(m)
    st = oracle.schedule(m)
    assert sum(len(x) for x in st) == N
    for sw in range(2):
        S, rec = oracle.sweep(m, S, sw)
    site = int(st[-1][-1])
    H, _ = oracle.cluster_hamiltonian(m, S, site, oracle.propose(m, 2, site, S[site]))
    e = oracle.eigvalsh(H)
    oracle.free_energy(e, m.mu, m.T)
    oracle.cluster_free_energy(m, S, site)
    oracle.in_window(m, site, 0)
    oracle.single_site_chain(m, S, site, 3, 20)
    oracle.structure_factor(m.Lx, m.Ly, S, np.pi, np.pi, Lz=m.Lz, qz=np.pi if m.Lz > 1 else 0.0)
for n in (1, 2, 17):
    oracle.eigvalsh(inputs.random_hermitian(n, n, scale=2.0))
oracle.philox4x32_10([1, 2], [3, 4, 5, 6])
oracle.uniform2(7, 8, 9, 2)
print("sanitized oracle ok")
"""


def test_oracle_is_clean_under_address_and_undefined_behaviour_sanitizers():
    libasan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(libasan) or not os.path.exists(libasan):
        pytest.skip("gcc has no AddressSanitizer runtime here")
    path = oracle.build(sanitize=True)
    env = dict(os.environ, LD_PRELOAD=libasan, PTCA_ORACLE_LIB=path,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1",
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", EXERCISE], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    report = r.stdout[-2000:] + r.stderr[-4000:]
    assert r.returncode == 0, report
    assert "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, report
    assert "sanitized oracle ok" in r.stdout, report


ABI_EXERCISE = r"""
import sys
import numpy as np
from paper_1502_07028_gb300 import _build
_build.LIB = sys.argv[1]
import paper_1502_07028_gb300 as P

assert P.ptca_version() == 1
good = [
    dict(Lx=8, Ly=8, L_c=4),
    dict(Lx=10, Ly=10, L_c=8, stride=5),
    dict(Lx=100, Ly=100, L_c=8, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=31, Ly=17, L_c=6, periodic=0, stride=6),
    dict(Lx=8, Ly=1, L_c=4, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=9, Ly=7, L_c=4, periodic=0, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=6, Ly=6, Lz=6, L_c=3, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=6, Ly=5, Lz=4, L_c=3, periodic=0, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=24, Ly=24, L_c=12, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=16, Ly=1, L_c=8, model=P.MODEL_HOLSTEIN, update_offset=4, stride=8),
    dict(Lx=8, Ly=8, Lz=8, L_c=4, model=P.MODEL_HUBBARD_MF, mu=4.0, schedule=P.SCHEDULE_BLOCK),
]
for kw in good:
    cfg = P.Config(**kw)
    st = P.ptca_schedule(cfg)
    assert sorted(np.concatenate(st).tolist()) == list(range(cfg.N))
    split = P.ptca_stage_split(cfg)
    assert len(split) == len(st)
bad = [
    dict(Lx=8, Ly=8, L_c=9),
    dict(Lx=8, Ly=8, L_c=4, stride=3),
    dict(Lx=8, Ly=8, L_c=4, model=3),
    dict(Lx=8, Ly=8, L_c=4, T=0.0),
    dict(Lx=8, Ly=1, Lz=4, L_c=2),
    dict(Lx=40, Ly=40, L_c=17, schedule=P.SCHEDULE_BLOCK),
]
for kw in bad:
    try:
        P.ptca_schedule(P.Config(**kw))
    except P.PtcaError as e:
        assert e.status == 1 and str(e)
    else:
        raise AssertionError(kw)
try:
    P.ptca_init(P.Config(Lx=8, Ly=8, L_c=4))
except P.PtcaError as e:
    assert e.status == 2
else:
    raise AssertionError("ptca_init succeeded without a GPU")
print("sanitized abi ok")
"""


def test_host_side_of_the_c_abi_is_clean_under_sanitizers(tmp_path):
    # The ABI's host logic (validation, schedules, exactness check, stage
    # split, error reporting) lives in api.cu: rebuild that translation unit
    # with AddressSanitizer and UndefinedBehaviorSanitizer and link it with
    # the other objects of the normal build.  No GPU is touched.
    import torch
    from paper_1502_07028_gb300 import _build
    if torch.cuda.is_available():
        # The exercise relies on ptca_init failing for want of a device; with
        # a GPU it would create a context under the ASan runtime.
        pytest.skip("host-only check; a GPU is present")
    libasan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(libasan) or not os.path.exists(libasan):
        pytest.skip("gcc has no AddressSanitizer runtime here")
    _build.build()
    cc = _build.nvcc()
    san = "-fsanitize=address,-fsanitize=undefined,-fno-sanitize-recover=all,-fno-omit-frame-pointer"
    api_o = str(tmp_path / "api_san.o")
    lib = str(tmp_path / "libptca_san.so")
    subprocess.run([cc, *_build.ARCH, "-O1", "-g", "-std=c++17", "--expt-relaxed-constexpr",
                    "-Xcompiler", "-fPIC," + san, "-c", os.path.join(_build.CSRC, "api.cu"), "-o", api_o],
                   check=True, capture_output=True)
    objs = [os.path.join(_build.BUILD, s.replace(".cu", ".o")) for s in _build.SOURCES if s != "api.cu"]
    if not all(os.path.exists(o) for o in objs):
        _build.build(force=True)  # the library is current but its objects were removed
    subprocess.run([cc, *_build.ARCH, "-shared", "-Xcompiler", "-fsanitize=address,-fsanitize=undefined",
                    "-o", lib, api_o, *objs, "-lcudart"], check=True, capture_output=True)
    env = dict(os.environ, LD_PRELOAD=libasan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1:protect_shadow_gap=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1",
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", ABI_EXERCISE, lib], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    report = r.stdout[-2000:] + r.stderr[-4000:]
    assert r.returncode == 0, report
    assert "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, report
    assert "sanitized abi ok" in r.stdout, report
