"""Pins of the oracle on cubic lattices (Lz > 1): the paper's 3-D workloads
(Sec. IV and V: 4^3 traveling clusters, 2^3 = 8 blocks).  What the
mathematics fixes: ferromagnetic closed forms of periodic and open 4^3-type
clusters, the trace and Frobenius norm, invariance under a global spin
rotation, exact and covering 3-D schedules, and S(q) of ferromagnetic and
Neel states with its sum rule."""
import itertools
import math

import numpy as np
import pytest

import oracle
from tests import inputs


def _fm3_periodic(Lc, t, JH):
    k = [-2 * t * sum(math.cos(2 * math.pi * a / Lc) for a in ks) for ks in itertools.product(range(Lc), repeat=3)]
    return np.sort(np.array([e + s for e in k for s in (-JH, JH)]))


def _fm3_open(L, t, JH):
    c = [-2 * t * math.cos(math.pi * a / (L + 1)) for a in range(1, L + 1)]
    return np.sort(np.array([x + y + z + s for x in c for y in c for z in c for s in (-JH, JH)]))


def _m(**kw):
    base = dict(Lx=8, Ly=8, Lz=8, Lc=4, t=1.0, JH=8.0)
    base.update(kw)
    return oracle.Model(**base)


@pytest.mark.parametrize("Lc", [2, 3, 4])
def test_ferromagnet_periodic_cube_closed_form(Lc):
    m = _m(Lc=Lc)
    S = inputs.ferro_spins(m.N, (0.1, 0.5, -0.8))
    for site in (0, 77, m.N - 1):
        H, _ = oracle.cluster_hamiltonian(m, S, site)
        assert H.shape[0] == 2 * Lc ** 3
        assert np.max(np.abs(oracle.eigvalsh(H) - _fm3_periodic(Lc, 1.0, 8.0))) < 1e-12


def test_ferromagnet_open_cube_closed_form():
    m = _m(Lc=3, t=1.3, JH=5.0, cluster_periodic=0)
    S = inputs.ferro_spins(m.N, (0.0, 0.0, 1.0))
    H, _ = oracle.cluster_hamiltonian(m, S, 200)
    assert np.max(np.abs(oracle.eigvalsh(H) - _fm3_open(3, 1.3, 5.0))) < 1e-12


def test_open_lattice_clips_cube_windows():
    # 6^3 open lattice, L_c = 4, central offset 2: a corner window is 2x2x2.
    m = _m(Lx=6, Ly=6, Lz=6, Lc=4, lattice_periodic=0)
    S = inputs.ferro_spins(m.N, (1.0, 0.0, 0.0))
    H, _ = oracle.cluster_hamiltonian(m, S, 0)
    assert H.shape[0] == 2 * 8
    assert np.max(np.abs(oracle.eigvalsh(H) - _fm3_open(2, 1.0, 8.0))) < 1e-12


def test_trace_and_frobenius_norm_of_a_periodic_cube():
    # Random unit spins: tr H = 0 and ||H||_F^2 = N_c (2 J_H^2) + 12 N_c t^2
    # (three bonds per site, two spin species, both triangles).
    m = _m(Lc=4, t=1.1, JH=3.0)
    S = inputs.random_unit_spins(12, m.N)
    H, _ = oracle.cluster_hamiltonian(m, S, 101)
    Nc = 64
    assert abs(np.trace(H)) < 1e-12
    assert abs(np.sum(np.abs(H) ** 2) - (Nc * 2 * 9.0 + 12 * Nc * 1.21)) < 1e-9


def test_spectrum_invariant_under_a_global_rotation():
    m = _m(Lc=3)
    S = inputs.random_unit_spins(13, m.N)
    R = inputs.random_rotation(14)
    e1 = oracle.eigvalsh(oracle.cluster_hamiltonian(m, S, 55)[0])
    e2 = oracle.eigvalsh(oracle.cluster_hamiltonian(m, S @ R.T, 55)[0])
    assert np.max(np.abs(e1 - e2)) < 1e-11


def _sequentially_exact(m, stages):
    for st in stages:
        pos = {int(s): k for k, s in enumerate(st)}
        for k, b in enumerate(st):
            for g in st[:k]:
                if oracle.in_window(m, int(b), int(g)):
                    return False
    return True


@pytest.mark.parametrize("L,Lc,exact", [(6, 4, True), (6, 3, True), (8, 5, True), (6, 5, False)])
def test_block_schedule_has_eight_covering_stages(L, Lc, exact):
    m = _m(Lx=L, Ly=L, Lz=L, Lc=Lc, schedule=oracle.SCHEDULE_BLOCK)
    stages = oracle.schedule(m)
    assert len(stages) == 8
    flat = np.concatenate(stages)
    assert np.array_equal(np.sort(flat), np.arange(m.N))
    assert all(st.size == (L // 2) ** 3 for st in stages)
    assert _sequentially_exact(m, stages) == exact


def test_tiled_schedule_stages_are_mutually_independent():
    m = _m(Lx=8, Ly=8, Lz=8, Lc=4, stride=4)
    stages = oracle.schedule(m)
    assert len(stages) == 64 and all(st.size == 8 for st in stages)
    for st in stages:
        for a in st:
            for b in st:
                if a != b:
                    assert not oracle.in_window(m, int(a), int(b))


def test_structure_factor_ferro_neel_and_sum_rule():
    L = 4
    N = L ** 3
    S = inputs.ferro_spins(N, (0.3, 0.3, 0.9))
    assert abs(oracle.structure_factor(L, L, S, 0, 0, Lz=L, qz=0) - 1.0) < 1e-12
    idx = np.arange(N)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    neel = np.where((x + y + z) % 2 == 0, 1.0, -1.0)[:, None] * np.array([0.0, 0.0, 1.0])
    assert abs(oracle.structure_factor(L, L, neel, math.pi, math.pi, Lz=L, qz=math.pi) - 1.0) < 1e-12
    assert abs(oracle.structure_factor(L, L, neel, 0, 0, Lz=L, qz=0)) < 1e-12
    R = inputs.random_unit_spins(15, N)
    tot = sum(oracle.structure_factor(L, L, R, 2 * math.pi * a / L, 2 * math.pi * b / L, Lz=L,
                                      qz=2 * math.pi * c / L)
              for a in range(L) for b in range(L) for c in range(L))
    assert abs(tot - 1.0) < 1e-10   # sum over q of S(q) = (1/N) sum_i |S_i|^2
