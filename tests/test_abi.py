"""Host-side checks of the C ABI (no GPU): the library builds and loads,
exports every entry point include/ptca.h declares, builds the same stage
schedules as the oracle (Sec. III.a) and rejects invalid problems."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_1502_07028_gb300 as P
from paper_1502_07028_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    _build.build()
    return P.lib()


def _declared():
    names = []
    with open(os.path.join(ROOT, "include", "ptca.h")) as f:
        text = f.read()
    for m in re.finditer(r"^\s*(?:const\s+char\s*\*|ptca_status|int32_t)\s+(ptca_\w+)\s*\(", text, re.M):
        names.append(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ptca_init", "ptca_build_clusters", "ptca_cluster_eigvals", "ptca_free_energy",
                     "ptca_sweep", "ptca_observables"):
        assert required in names
    assert sorted(names) == sorted(P.ptca.EXPORTED)


def test_binding_has_a_same_named_function_for_every_entry_point(built):
    for name in _declared():
        assert callable(getattr(P, name, None)), name
    P.lib().ptca_version()
    assert isinstance(P.ptca_last_error(), str)


def test_library_exports_every_declared_symbol(built):
    for name in _declared():
        assert hasattr(built, name), name
    assert P.ptca_version() == 1


def test_symbols_are_c_linkage(built):
    # extern "C": plain names resolve through dlsym.
    dl = ctypes.CDLL(_build.LIB)
    for name in _declared():
        assert ctypes.cast(getattr(dl, name), ctypes.c_void_p).value


@pytest.mark.parametrize("kw", [
    dict(Lx=8, Ly=8, L_c=4),
    dict(Lx=10, Ly=10, L_c=8, stride=5),
    dict(Lx=32, Ly=32, L_c=8, stride=8),
    dict(Lx=12, Ly=12, L_c=4, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=100, Ly=100, L_c=8, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=31, Ly=17, L_c=6, periodic=0, stride=6),
    dict(Lx=8, Ly=1, L_c=4, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=9, Ly=7, L_c=4, periodic=0, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=8, Ly=8, Lz=8, L_c=4, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=6, Ly=6, Lz=6, L_c=3, stride=3),
    dict(Lx=7, Ly=6, Lz=5, L_c=3, periodic=0, schedule=P.SCHEDULE_BLOCK),
])
def test_schedule_matches_oracle(built, kw):
    cfg = P.Config(**kw)
    mine = P.ptca_schedule(cfg)
    m = oracle.Model(Lx=cfg.Lx, Ly=cfg.Ly, Lz=cfg.Lz, Lc=cfg.L_c, lattice_periodic=cfg.periodic,
                     schedule=cfg.schedule, stride=cfg.stride)
    ref = oracle.schedule(m)
    assert len(mine) == len(ref)
    for a, b in zip(mine, ref):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("kw,why", [
    (dict(Lx=8, Ly=8, L_c=4, stride=2), "not exact"),
    (dict(Lx=10, Ly=10, L_c=4, stride=3), "divide"),
    (dict(Lx=8, Ly=8, L_c=1), "L_c"),
    (dict(Lx=8, Ly=8, L_c=9), "L_c"),
    (dict(Lx=12, Ly=12, L_c=8, schedule=P.SCHEDULE_BLOCK), "not exact"),
    (dict(Lx=8, Ly=8, L_c=4, T=0.0), "T > 0"),
    (dict(Lx=68, Ly=68, L_c=17, precision=P.MIXED), "maximum"),
    (dict(Lx=56, Ly=56, Lz=7, L_c=7, precision=P.MIXED), "maximum"),
    (dict(Lx=8, Ly=8, L_c=4, update_offset=4), "update_offset"),
    (dict(Lx=8, Ly=1, Lz=4, L_c=2), "needs Ly > 1"),
    (dict(Lx=8, Ly=8, L_c=4, model=3), "unknown model"),
    (dict(Lx=8, Ly=8, L_c=4, model=P.MODEL_HUBBARD_MF, m_step=0.0), "m_step"),
    (dict(Lx=8, Ly=8, L_c=4, model=P.MODEL_HUBBARD_MF, U=float("nan")), "finite U"),
    (dict(Lx=16, Ly=1, L_c=4, model=P.MODEL_HOLSTEIN, lam=float("inf")), "finite lambda"),
    (dict(Lx=16, Ly=1, L_c=4, model=P.MODEL_HOLSTEIN, m_step=-1.0), "m_step"),
    (dict(Lx=8, Ly=8, Lz=3, L_c=4), "L_c"),
    (dict(Lx=8, Ly=8, Lz=6, L_c=4, stride=4), "divide"),
])
def test_invalid_problems_are_rejected(built, kw, why):
    with pytest.raises(P.PtcaError) as e:
        P.ptca_schedule(P.Config(**kw))
    assert e.value.status == 1
    assert why in str(e.value)


def test_init_reports_missing_gpu_instead_of_falling_back(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.PtcaError) as e:
        P.ptca_init(P.Config(Lx=8, Ly=8, L_c=4))
    assert e.value.status == 2


def test_binding_fails_loudly_without_the_library(built, monkeypatch, tmp_path):
    # No silent substitute: a missing shared library is an error on every call.
    monkeypatch.setattr(P.ptca, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "libptca.so"))
    with pytest.raises(RuntimeError, match="is missing"):
        P.ptca_version()
    with pytest.raises(RuntimeError, match="is missing"):
        P.ptca_init(P.Config(Lx=8, Ly=8, L_c=4))


@pytest.mark.parametrize("kw", [
    dict(Lx=8, Ly=8, L_c=4),
    dict(Lx=10, Ly=10, L_c=8, stride=5),
    dict(Lx=32, Ly=32, L_c=8, stride=8),
    dict(Lx=12, Ly=12, L_c=4, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=31, Ly=17, L_c=6, periodic=0, stride=6),
    dict(Lx=8, Ly=1, L_c=4, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=9, Ly=7, L_c=4, periodic=0, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=6, Ly=6, Lz=6, L_c=3, schedule=P.SCHEDULE_BLOCK),
    dict(Lx=6, Ly=5, Lz=4, L_c=3, periodic=0, schedule=P.SCHEDULE_BLOCK),
])
def test_stage_split_follows_the_window_rule(built, kw):
    """The overlapped pipeline's split, against the oracle's window rule
    (Sec. II.b): a visit of stage s is independent iff no site of stage s-1
    (cyclically) lies in its window; each part is ordered largest window
    first, ties in schedule order."""
    cfg = P.Config(**kw)
    m = oracle.Model(Lx=cfg.Lx, Ly=cfg.Ly, Lz=cfg.Lz, Lc=cfg.L_c, lattice_periodic=cfg.periodic,
                     schedule=cfg.schedule, stride=cfg.stride)
    stages = oracle.schedule(m)
    split = P.ptca_stage_split(cfg)
    assert len(split) == len(stages)
    N = cfg.N
    wsize = {}
    for s, sites in enumerate(stages):
        prev = stages[(s - 1) % len(stages)]
        dep = []
        for c, site in enumerate(sites):
            dep.append(any(oracle.in_window(m, int(site), int(q)) for q in prev))
            if int(site) not in wsize:
                wsize[int(site)] = sum(oracle.in_window(m, int(site), g) for g in range(N))
        order, n_indep = split[s]
        assert sorted(order.tolist()) == list(range(sites.size))
        assert n_indep == dep.count(False)
        for part in (order[:n_indep], order[n_indep:]):
            key = [(-wsize[int(sites[c])], int(c)) for c in part]
            assert key == sorted(key)
        assert not any(dep[c] for c in order[:n_indep])
        assert all(dep[c] for c in order[n_indep:])


def test_stage_split_of_the_100x100_block_schedule(built):
    """Block schedule, 100 x 100 torus, L_c = 8, windows [x, x+7] x [y, y+7]:
    a quadrant's visits that depend on the quadrant before it are the 7
    columns whose windows wrap or reach into it (7 x 50 = 350), or, for the
    quadrant diagonal to it, a 7 x 7 corner (49)."""
    cfg = P.Config(Lx=100, Ly=100, L_c=8, schedule=P.SCHEDULE_BLOCK, precision=P.MIXED)
    split = P.ptca_stage_split(cfg)
    assert [n for _, n in split] == [2500 - 49, 2500 - 350, 2500 - 49, 2500 - 350]


def test_stage_split_of_the_benchmarked_cube_large_cluster_and_chain_workloads(built):
    """Closed forms of the split for the other benchmarked workloads.  With
    corner windows [x, x+L_c-1] (block schedule), a visit depends on the
    previous block iff, along every axis where the two blocks differ, it lies
    within L_c-1 of its half's end: (L_c-1) of the half's positions on such
    an axis, all of them on the others."""
    # 40^3 torus, 4^3 clusters: blocks of 20^3 in the order (bz, by, bx).
    cube = P.ptca_stage_split(P.Config(Lx=40, Ly=40, Lz=40, L_c=4, schedule=P.SCHEDULE_BLOCK,
                                       model=P.MODEL_HUBBARD_MF, mu=4.0, precision=P.MIXED))
    differ = [3, 1, 2, 1, 3, 1, 2, 1]     # axes in which block s and block s-1 differ
    assert [n for _, n in cube] == [8000 - 3 ** d * 20 ** (3 - d) for d in differ]
    # 48^2 torus, 12^2 clusters (matrix order 288): blocks of 24^2.
    large = P.ptca_stage_split(P.Config(Lx=48, Ly=48, L_c=12, schedule=P.SCHEDULE_BLOCK, precision=P.MIXED))
    assert [n for _, n in large] == [576 - 121, 576 - 11 * 24, 576 - 121, 576 - 11 * 24]
    # Holstein chain with the central update site (tiled, stride N_c = 8):
    # every window [c-4, c+3] holds c-1, a site of the previous stage.
    chain = P.ptca_stage_split(P.Config(Lx=65536, Ly=1, L_c=8, schedule=P.SCHEDULE_TILED, stride=8,
                                        update_offset=4, model=P.MODEL_HOLSTEIN, lam=1.5, K=1.0, mu=0.0,
                                        m_step=0.4, precision=P.MIXED))
    assert len(chain) == 8 and all(n == 0 for _, n in chain)


@pytest.mark.parametrize("Lc", [11, 12, 16])
def test_large_clusters_are_accepted(built, Lc):
    # Orders above the shared-memory kernels' (2 N_c = 242, 288, 512) go to
    # the large-cluster path; the schedule is the same rule.
    stages = P.ptca_schedule(P.Config(Lx=2 * Lc, Ly=2 * Lc, L_c=Lc, schedule=P.SCHEDULE_BLOCK, precision=P.MIXED))
    assert len(stages) == 4 and sum(st.size for st in stages) == 4 * Lc * Lc


def test_binding_structs_match_the_header_layout(tmp_path):
    # gcc compiles include/ptca.h as C and prints each struct's size and field
    # offsets; the ctypes mirrors must agree field by field.
    structs = {"ptca_lattice": P.ptca.Lattice, "ptca_params": P.ptca.Params,
               "ptca_sweep_stats": P.ptca.SweepStats, "ptca_obs": P.ptca.Obs,
               "ptca_launch_config": P.ptca.LaunchConfig}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "ptca.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    # Strict C99: the header is plain C, usable from any C toolchain.
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_noalloc_validates_on_the_host_before_touching_the_device(built):
    # Every check of ptca_sweep_noalloc runs on the host before its first CUDA
    # call: without a GPU a valid call stops at the device lookup (status 2),
    # every invalid one earlier (status 1).  The device pointers are dummies
    # that nothing dereferences on the host.  The binding's own checks want
    # CUDA tensors, so the C entry point is called directly.
    import ctypes

    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    dummy = ctypes.c_void_p(0x1000)

    def status(cfg=P.Config(Lx=8, Ly=8, L_c=4), spins=dummy, sweep_index=0):
        lat, par = cfg.lattice(), cfg.params()
        st = P.lib().ptca_sweep_noalloc(ctypes.byref(lat), ctypes.byref(par), spins, sweep_index, dummy, dummy,
                                        dummy, None)
        return st, P.lib().ptca_last_error().decode()

    st, msg = status()
    assert st == 2 and "device" in msg
    assert status(sweep_index=-1)[0] == 1
    assert status(spins=None)[0] == 1
    st, msg = status(cfg=P.Config(Lx=200, Ly=200, L_c=4))
    assert st == 1 and "at most 16384" in msg
    assert status(cfg=P.Config(Lx=8, Ly=8, L_c=9))[0] == 1
    assert status(cfg=P.Config(Lx=8, Ly=8, L_c=4, model=P.MODEL_HOLSTEIN, m_step=0.0))[0] == 1


def test_noalloc_binding_checks_its_tensors(built):
    # The binding refuses anything but contiguous CUDA tensors of the right
    # dtype and size before it reaches the library.
    import torch
    cfg = P.Config(Lx=8, Ly=8, L_c=4)
    with pytest.raises(ValueError, match="CUDA"):
        P.ptca_sweep_noalloc(cfg, torch.zeros((cfg.N, 3), dtype=torch.float64), 0)
    with pytest.raises(ValueError):
        P.ptca_sweep_noalloc(cfg, None, 0)


def test_smoke_refuses_to_run_without_a_gpu(built):
    # The smoke check exercises the CUDA path only; without a device it
    # fails instead of falling back to anything.
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import __graft_entry__
    with pytest.raises(RuntimeError, match="cuda:0"):
        __graft_entry__.smoke()
