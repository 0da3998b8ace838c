"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: every expected value is a
closed form, a published known-answer vector, a library routine used as an
independent cross-check (LAPACK via numpy, scipy's matrix exponential), a
brute-force many-body calculation, or a structural count printed in the paper.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from tests import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Counter-based generator (Philox4x32-10, published known-answer vectors)
# --------------------------------------------------------------------------
def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    out = oracle.philox4x32_10(key, ctr)
    assert [int(x) for x in out] == expect


def test_uniforms_open_interval_and_moments():
    u = np.array([oracle.uniform2(7, s, i, p) for s in range(3) for i in range(400) for p in range(3)])
    assert u.min() > 0.0 and u.max() < 1.0
    flat = u.ravel()
    n = flat.size
    assert abs(flat.mean() - 0.5) < 4 * math.sqrt(1 / 12 / n)
    assert abs(flat.var() - 1 / 12) < 0.01
    # Distinct purposes give distinct streams.
    assert not np.allclose(oracle.uniform2(7, 0, 0, 0), oracle.uniform2(7, 0, 0, 1))


# --------------------------------------------------------------------------
# Initial spins and proposals (Sec. II.c step c)
# --------------------------------------------------------------------------
def test_init_spins_uniform_on_sphere():
    m = oracle.Model(Lx=100, Ly=100, Lc=4)
    S = oracle.init_spins(m)
    assert np.allclose(np.linalg.norm(S, axis=1), 1.0, atol=1e-14)
    n = S.shape[0]
    assert np.all(np.abs(S.mean(axis=0)) < 4 * math.sqrt(1 / 3 / n))
    assert np.all(np.abs((S ** 2).mean(axis=0) - 1 / 3) < 0.02)


@pytest.mark.parametrize("s_old", [(0, 0, 1), (0, 0, -1), (1, 0, 0), (0.3, -0.5, 0.81)])
def test_cone_proposal_stays_in_cap_and_is_uniform_on_it(s_old):
    s_old = np.asarray(s_old, float) / np.linalg.norm(s_old)
    m = oracle.Model(Lx=64, Ly=64, Lc=4, proposal=oracle.PROPOSAL_CONE, cone_deg=30.0, seed=3)
    props = []
    for site in range(3000):
        s = oracle.propose(m, 5, site, s_old)
        assert abs(np.linalg.norm(s) - 1.0) < 1e-14
        props.append(s)
    props = np.array(props)
    c = props @ s_old
    cmin = math.cos(math.radians(30.0))
    assert c.min() >= cmin - 1e-12
    # cos(theta) uniform on [cos 30deg, 1]: mean (1+cmin)/2, var (1-cmin)^2/12.
    sd = (1 - cmin) / math.sqrt(12 * c.size)
    assert abs(c.mean() - (1 + cmin) / 2) < 5 * sd
    # Azimuth uniform about s_old: the part perpendicular to s_old averages to
    # zero, each of its components with variance E[sin^2 theta]/2.
    perp = props - c[:, None] * s_old
    sd_perp = math.sqrt(np.mean(np.sum(perp ** 2, axis=1)) / 2 / c.size)
    assert np.all(np.abs(perp.mean(axis=0)) < 5 * sd_perp)


def test_sphere_proposal_ignores_old_spin_and_is_isotropic():
    m = oracle.Model(Lx=64, Ly=64, Lc=4, proposal=oracle.PROPOSAL_SPHERE, seed=11)
    P = np.array([oracle.propose(m, 2, i, (0, 0, 1)) for i in range(4000)])
    Q = np.array([oracle.propose(m, 2, i, (1, 0, 0)) for i in range(4000)])
    assert np.array_equal(P, Q)
    assert np.all(np.abs(P.mean(axis=0)) < 4 * math.sqrt(1 / 3 / 4000))


# --------------------------------------------------------------------------
# Cluster Hamiltonian (Sec. II.b-c, Fig. 1; double-exchange model)
# --------------------------------------------------------------------------
def _fm_periodic(Lc, t, JH):
    k = [-2 * t * (math.cos(2 * math.pi * a / Lc) + math.cos(2 * math.pi * b / Lc))
         for a in range(Lc) for b in range(Lc)]
    return np.sort(np.array([e + s for e in k for s in (-JH, JH)]))


def _fm_open(ex, ey, t, JH):
    kx = [-2 * t * math.cos(math.pi * a / (ex + 1)) for a in range(1, ex + 1)]
    ky = [-2 * t * math.cos(math.pi * b / (ey + 1)) for b in range(1, ey + 1)] if ey > 1 else [0.0]
    return np.sort(np.array([x + y + s for x in kx for y in ky for s in (-JH, JH)]))


@pytest.mark.parametrize("Lc", [2, 3, 4, 5])
def test_ferromagnet_periodic_cluster_closed_form(Lc):
    m = oracle.Model(Lx=8, Ly=8, Lc=Lc, t=1.0, JH=8.0)
    S = inputs.ferro_spins(m.N, (0.2, -0.7, 0.4))
    for site in (0, 9, 63):
        H, (ex, ey) = oracle.cluster_hamiltonian(m, S, site)
        assert (ex, ey) == (Lc, Lc)
        e = oracle.eigvalsh(H)
        assert np.max(np.abs(e - _fm_periodic(Lc, 1.0, 8.0))) < 1e-12


@pytest.mark.parametrize("Lc", [2, 3, 4, 6])
def test_ferromagnet_open_cluster_closed_form(Lc):
    m = oracle.Model(Lx=8, Ly=8, Lc=Lc, t=1.3, JH=6.0, cluster_periodic=0)
    S = inputs.ferro_spins(m.N, (1.0, 1.0, -0.5))
    H, _ = oracle.cluster_hamiltonian(m, S, 20)
    e = oracle.eigvalsh(H)
    assert np.max(np.abs(e - _fm_open(Lc, Lc, 1.3, 6.0))) < 1e-12


def test_open_lattice_clips_windows_to_rectangles():
    # 10x10 open lattice, L_c = 10, update site at offset 5 (window c-5..c+4):
    # clipped to 5 sites at the low edge, 6 at the high edge (open boundary).
    m = oracle.Model(Lx=10, Ly=10, Lc=10, t=1.0, JH=6.0, lattice_periodic=0)
    S = inputs.ferro_spins(m.N, (0, 0, 1))
    for site, shape in ((0, (5, 5)), (5, (10, 5)), (99, (6, 6)), (55, (10, 10)), (9, (6, 5))):
        H, (ex, ey) = oracle.cluster_hamiltonian(m, S, site)
        assert (ex, ey) == shape
        e = oracle.eigvalsh(H)
        assert np.max(np.abs(e - _fm_open(ex, ey, 1.0, 6.0))) < 1e-12


def test_chain_periodic_cluster_closed_form():
    m = oracle.Model(Lx=8, Ly=1, Lc=4, t=1.0, JH=2.0)
    S = inputs.ferro_spins(m.N, (0, 1, 0))
    H, (ex, ey) = oracle.cluster_hamiltonian(m, S, 3)
    assert (ex, ey) == (4, 1)
    k = [-2 * math.cos(2 * math.pi * a / 4) for a in range(4)]
    expect = np.sort([x + s for x in k for s in (-2.0, 2.0)])
    assert np.max(np.abs(oracle.eigvalsh(H) - expect)) < 1e-12


def test_trace_zero_and_frobenius_closed_form():
    for Lc in (3, 4, 8):
        m = oracle.Model(Lx=16, Ly=16, Lc=Lc, t=1.0, JH=8.0)
        S = inputs.random_unit_spins(1, m.N)
        H, _ = oracle.cluster_hamiltonian(m, S, 37)
        assert np.allclose(H, H.conj().T, atol=0)
        assert abs(np.trace(H)) < 1e-12
        Nc = Lc * Lc
        assert abs(np.sum(np.abs(H) ** 2) - Nc * (2 * 8.0 ** 2 + 8 * 1.0 ** 2)) < 1e-9


def test_zero_hopping_gives_plus_minus_JH():
    m = oracle.Model(Lx=6, Ly=6, Lc=3, t=0.0, JH=5.0)
    S = inputs.random_unit_spins(2, m.N)
    e = oracle.eigvalsh(oracle.cluster_hamiltonian(m, S, 7)[0])
    assert np.max(np.abs(e - np.array([-5.0] * 9 + [5.0] * 9))) < 1e-12


def test_spectrum_invariant_under_global_spin_rotation():
    m = oracle.Model(Lx=8, Ly=8, Lc=4)
    S = inputs.random_unit_spins(3, m.N)
    R = inputs.random_rotation(4)
    e1 = oracle.eigvalsh(oracle.cluster_hamiltonian(m, S, 27)[0])
    e2 = oracle.eigvalsh(oracle.cluster_hamiltonian(m, S @ R.T, 27)[0])
    assert np.max(np.abs(e1 - e2)) < 1e-12


def test_window_equal_to_lattice_is_translation_invariant():
    # With L_c = L on a torus the periodic cluster is the whole system
    # (Sec. II.b: the cluster spectrum becomes the system's); every update
    # site then sees the same spectrum.
    m = oracle.Model(Lx=4, Ly=4, Lc=4)
    S = inputs.random_unit_spins(5, m.N)
    ref = oracle.eigvalsh(oracle.cluster_hamiltonian(m, S, 0)[0])
    for site in (1, 6, 15):
        e = oracle.eigvalsh(oracle.cluster_hamiltonian(m, S, site)[0])
        assert np.max(np.abs(e - ref)) < 1e-12


def test_replacing_update_spin_changes_only_its_block():
    m = oracle.Model(Lx=8, Ly=8, Lc=4, JH=8.0)
    S = inputs.random_unit_spins(6, m.N)
    site = 18
    s_new = np.array([0.6, 0.0, -0.8])
    H0, (ex, _) = oracle.cluster_hamiltonian(m, S, site)
    H1, _ = oracle.cluster_hamiltonian(m, S, site, s_new)
    D = H1 - H0
    w = 2 * ex + 2  # update site sits at window position (2, 2)
    blk = D[2 * w:2 * w + 2, 2 * w:2 * w + 2]
    ds = s_new - S[site]
    expect = -8.0 * np.array([[ds[2], ds[0] - 1j * ds[1]], [ds[0] + 1j * ds[1], -ds[2]]])
    assert np.allclose(blk, expect, atol=1e-14)
    D[2 * w:2 * w + 2, 2 * w:2 * w + 2] = 0
    assert np.max(np.abs(D)) == 0.0


# --------------------------------------------------------------------------
# Jacobi eigensolver (cross-checked against LAPACK through numpy)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 8, 33, 64])
def test_jacobi_matches_lapack(n):
    H = inputs.random_hermitian(100 + n, n, scale=3.0)
    e = oracle.eigvalsh(H)
    ref = np.linalg.eigvalsh(H)
    assert np.max(np.abs(e - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))
    fro2 = np.sum(np.abs(H) ** 2)
    assert abs(e.sum() - np.trace(H).real) < 1e-13 * n * math.sqrt(fro2)
    assert abs(np.sum(e ** 2) - fro2) < 1e-13 * fro2


def _cluster_cases():
    """Physical cluster matrices of order 8 and 16, degenerate spectra included."""
    cases = []
    m = oracle.Model(Lx=4, Ly=4, Lc=2, t=1.0, JH=8.0)
    cases.append(oracle.cluster_hamiltonian(m, inputs.random_unit_spins(21, m.N), 5)[0])
    cases.append(oracle.cluster_hamiltonian(m, inputs.ferro_spins(m.N, (0.3, -0.4, 0.866)), 5)[0])
    mh = oracle.Model(Lx=6, Ly=6, Lc=2, t=1.0, U=8.0, mu=4.0, model=oracle.MODEL_HUBBARD_MF, m_step=0.5)
    cases.append(oracle.cluster_hamiltonian(mh, inputs.random_fields(22, mh.N, 2.0), 7)[0])
    mq = oracle.Model(Lx=16, Ly=1, Lc=4, t=1.0, lam=1.5, K=1.0, model=oracle.MODEL_HOLSTEIN, m_step=0.4)
    S = np.zeros((mq.N, 3))
    S[:, 0] = inputs.rng(23).uniform(-1, 1, size=mq.N)
    cases.append(oracle.cluster_hamiltonian(mq, S, 6)[0])
    mc = oracle.Model(Lx=4, Ly=4, Lz=4, Lc=2, t=1.0, JH=6.0)
    cases.append(oracle.cluster_hamiltonian(mc, inputs.random_unit_spins(24, mc.N), 21)[0])
    return cases


@pytest.mark.parametrize("case", range(5))
def test_jacobi_spectrum_has_the_power_sums_of_the_cluster_matrix(case):
    # Newton's identities: the power sums p_k = sum_j eps_j^k = Tr(H^k),
    # k = 1..n, fix the characteristic polynomial and so the whole spectrum
    # with multiplicities.  The traces come from plain matrix products, with
    # no eigensolver involved.
    H = _cluster_cases()[case]
    n = H.shape[0]
    assert n in (8, 16)
    e = oracle.eigvalsh(H)
    assert np.all(np.diff(e) >= 0)
    P = np.eye(n, dtype=np.complex128)
    for k in range(1, n + 1):
        P = P @ H
        tr = np.trace(P)
        scale = float(np.sum(np.abs(e) ** k))
        assert abs(tr.imag) <= 1e-12 * scale
        assert abs(np.sum(e ** k) - tr.real) <= 1e-12 * scale, (k, np.sum(e ** k), tr)


def test_jacobi_special_matrices():
    assert np.array_equal(oracle.eigvalsh(np.zeros((5, 5))), np.zeros(5))
    d = np.array([3.0, -1.0, 2.0, 2.0])
    assert np.array_equal(oracle.eigvalsh(np.diag(d)), np.sort(d))
    # 2x2 closed form (a+b)/2 -+ sqrt(((a-b)/2)^2 + |z|^2).
    a, b, z = 1.5, -0.25, 0.3 - 0.7j
    r = math.sqrt(((a - b) / 2) ** 2 + abs(z) ** 2)
    e = oracle.eigvalsh(np.array([[a, z], [np.conj(z), b]]))
    assert np.allclose(e, [(a + b) / 2 - r, (a + b) / 2 + r], atol=1e-15, rtol=0)


# --------------------------------------------------------------------------
# Free energy (grand-canonical one-body formula)
# --------------------------------------------------------------------------
def _fock_grand_potential(H, mu, T):
    """-T ln Tr exp(-(H_mb - mu N)/T) over the full Fock space, brute force."""
    n = H.shape[0]
    dim = 1 << n
    K = np.zeros((dim, dim), dtype=np.complex128)
    for s in range(dim):
        for a in range(n):
            for b in range(n):
                if H[a, b] == 0 or not (s >> b) & 1:
                    continue
                sign = (-1) ** bin(s & ((1 << b) - 1)).count("1")
                s1 = s ^ (1 << b)
                if (s1 >> a) & 1:
                    continue
                sign *= (-1) ** bin(s1 & ((1 << a) - 1)).count("1")
                K[s1 | (1 << a), s] += sign * H[a, b]
        K[s, s] -= mu * bin(s).count("1")
    k = np.linalg.eigvalsh(K)
    x = -k / T
    xm = x.max()
    return -T * (xm + math.log(np.exp(x - xm).sum()))


def test_free_energy_equals_many_body_grand_potential_2x2():
    m = oracle.Model(Lx=4, Ly=4, Lc=2, t=1.0, JH=3.0)
    S = inputs.random_unit_spins(7, m.N)
    H, _ = oracle.cluster_hamiltonian(m, S, 5)
    assert H.shape == (8, 8)
    for mu, T in ((-1.0, 0.5), (0.3, 0.2), (-3.5, 1.0)):
        F = oracle.free_energy(oracle.eigvalsh(H), mu, T)
        assert abs(F - _fock_grand_potential(H, mu, T)) < 1e-11


def test_free_energy_equals_log_det_3x3():
    from scipy.linalg import expm
    m = oracle.Model(Lx=6, Ly=6, Lc=3, t=1.0, JH=8.0)
    S = inputs.random_unit_spins(8, m.N)
    H, _ = oracle.cluster_hamiltonian(m, S, 14)
    # scipy's scaling-and-squaring stays accurate while ||H - mu||/T is a
    # few hundred at most, hence the moderate temperatures.
    for mu, T in ((-6.5, 0.5), (-6.5, 1.0), (-2.0, 0.7)):
        E = expm(-(H - mu * np.eye(H.shape[0])) / T)
        sign, logdet = np.linalg.slogdet(np.eye(H.shape[0]) + E)
        assert abs(sign - 1) < 1e-9
        F = oracle.free_energy(oracle.eigvalsh(H), mu, T)
        assert abs(F - (-T * logdet)) < 1e-11 * abs(F)


def test_free_energy_limits():
    e = np.array([-3.0, -1.0, 0.5, 2.0])
    # T -> 0: sum of (eps - mu) over occupied levels.
    F0 = oracle.free_energy(e, 0.0, 1e-4)
    assert abs(F0 - (-4.0)) < 4 * 1e-4 * math.log(2)
    # mu -> -inf: F -> -T sum exp(-(eps - mu)/T) -> 0.
    mu, T = -60.0, 2.0
    F = oracle.free_energy(e, mu, T)
    series = -T * np.sum(np.exp(-(e - mu) / T))
    assert abs(F - series) < 1e-12 * abs(series)
    # Large beta stays finite (no overflow in exp).
    assert math.isfinite(oracle.free_energy(e, 5.0, 1e-3))


# --------------------------------------------------------------------------
# Schedules (Sec. III.a, Fig. 3)
# --------------------------------------------------------------------------
def _golden_fig3():
    d = {}
    with open(os.path.join(GOLDEN, "fig3_chain_counts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            d[k] = int(v)
    return d


def test_fig3_independent_and_boundary_cluster_counts():
    g = _golden_fig3()
    m = oracle.Model(Lx=g["N"], Ly=1, Lc=g["Nc"], schedule=oracle.SCHEDULE_BLOCK)
    # Sequential sweep 0..N-1 with the update site at the left end (ox = 0):
    # a cluster is a boundary cluster when it contains an earlier-visited site.
    boundary = sum(any(oracle.in_window(m, j, i) for i in range(j)) for j in range(g["N"]))
    assert boundary == g["boundary"]
    assert g["N"] - boundary == g["independent"]
    stages = oracle.schedule(m)
    assert len(stages) == g["blocks"]
    assert all(len(s) == g["block_size"] for s in stages)


def _sequentially_exact(m, stages):
    """Within each stage no site is inside the window of a later site."""
    for st in stages:
        for a, b in itertools.combinations(list(st), 2):
            if oracle.in_window(m, int(b), int(a)):
                return False
    return True


def _mutually_independent(m, stages):
    for st in stages:
        for a, b in itertools.combinations(list(st), 2):
            if oracle.in_window(m, int(b), int(a)) or oracle.in_window(m, int(a), int(b)):
                return False
    return True


def _covers_once(m, stages):
    flat = np.concatenate(stages)
    return flat.size == m.N and np.array_equal(np.sort(flat), np.arange(m.N))


@pytest.mark.parametrize("L,Lc", [(8, 4), (8, 5), (12, 4), (12, 7), (10, 6)])
def test_block_schedule_exact_iff_Lc_at_most_half_plus_one(L, Lc):
    m = oracle.Model(Lx=L, Ly=L, Lc=Lc, schedule=oracle.SCHEDULE_BLOCK)
    stages = oracle.schedule(m)
    assert len(stages) == 4 and _covers_once(m, stages)
    assert _sequentially_exact(m, stages) == (Lc <= L // 2 + 1)


@pytest.mark.parametrize("L,Lc,s", [(8, 4, 2), (8, 4, 4), (12, 4, 3), (12, 5, 3), (16, 8, 4),
                                    (20, 8, 5), (20, 8, 4), (10, 8, 10)])
def test_tiled_schedule_independent_iff_stride_clears_window(L, Lc, s):
    m = oracle.Model(Lx=L, Ly=L, Lc=Lc, schedule=oracle.SCHEDULE_TILED, stride=s)
    stages = oracle.schedule(m)
    assert len(stages) == s * s and _covers_once(m, stages)
    o = Lc // 2
    assert _mutually_independent(m, stages) == (s >= max(o + 1, Lc - o))


def test_sequential_sweep_equals_stagewise_snapshot_sweep():
    # PTCA's claim (Sec. III.a): clusters of one stage may be diagonalised at
    # once from the stage-start configuration.  Emulate that and compare with
    # the oracle's one-visit-at-a-time sweep, for both schedule kinds.
    for sched, stride in ((oracle.SCHEDULE_BLOCK, 0), (oracle.SCHEDULE_TILED, 4)):
        m = oracle.Model(Lx=8, Ly=8, Lc=4, T=0.5, mu=-6.5, schedule=sched, stride=stride, seed=9)
        S0 = oracle.init_spins(m)
        S_seq, rec = oracle.sweep(m, S0, 0)
        S = S0.copy()
        for st in oracle.schedule(m):
            snap = S.copy()
            for site in st:
                site = int(site)
                F_old = oracle.cluster_free_energy(m, snap, site)
                s_new = oracle.propose(m, 0, site, snap[site])
                F_new = oracle.cluster_free_energy(m, snap, site, s_new)
                u = oracle.uniform2(m.seed, 0, site, 2)[0]
                if math.log(u) < -(F_new - F_old) / m.T:
                    S[site] = s_new
        assert np.array_equal(S, S_seq)
        assert 0 < rec.accepted.sum() < m.N


@pytest.mark.parametrize("kw", [
    dict(Lx=6, Ly=6, Lz=6, Lc=3, schedule=oracle.SCHEDULE_BLOCK, T=0.5),               # cube, 8 blocks
    dict(Lx=5, Ly=4, Lz=3, Lc=3, lattice_periodic=0, schedule=oracle.SCHEDULE_BLOCK),  # open box
    dict(Lx=8, Ly=8, Lc=4, model=oracle.MODEL_HUBBARD_MF, U=8.0, mu=4.0, T=0.2, schedule=oracle.SCHEDULE_BLOCK),
    dict(Lx=32, Ly=1, Lc=8, model=oracle.MODEL_HOLSTEIN, lam=1.5, K=1.0, mu=0.0, T=0.1, m_step=0.4,
         schedule=oracle.SCHEDULE_TILED, stride=8, ox=4),                               # central site
])
def test_stagewise_snapshot_sweep_for_every_model_and_dimension(kw):
    # The same PTCA claim for cubic lattices and for the Hubbard and Holstein
    # models, whose cluster free energies carry a classical term.
    m = oracle.Model(**{"t": 1.0, "seed": 11, **kw})
    S0 = oracle.init_spins(m)
    S_seq, rec = oracle.sweep(m, S0, 3)
    S = S0.copy()
    for st in oracle.schedule(m):
        snap = S.copy()
        for site in st:
            site = int(site)
            F_old = oracle.cluster_free_energy(m, snap, site)
            s_new = oracle.propose(m, 3, site, snap[site])
            F_new = oracle.cluster_free_energy(m, snap, site, s_new)
            u = oracle.uniform2(m.seed, 3, site, 2)[0]
            if math.log(u) < -(F_new - F_old) / m.T:
                S[site] = s_new
    assert np.array_equal(S, S_seq)
    assert 0 < rec.accepted.sum() < m.N


# --------------------------------------------------------------------------
# Metropolis (Sec. II.c steps e-f): stationary distribution of one site
# --------------------------------------------------------------------------
def test_single_site_chain_samples_boltzmann_weight_of_cluster_free_energy():
    # All spins frozen except one; sphere proposals are symmetric, so the
    # chain must sample p(S) ~ exp(-F(S)/T) over the unit sphere.  Compare
    # the histogram of S_z with the marginal from quadrature of exp(-F/T).
    m = oracle.Model(Lx=4, Ly=4, Lc=2, t=1.0, JH=2.0, mu=-1.0, T=0.15, seed=21)
    S = inputs.ferro_spins(m.N, (0, 0, 1))
    site = 5
    nz, nphi = 48, 24
    zs = -1 + (np.arange(nz) + 0.5) * 2 / nz
    phis = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    logw = np.zeros(nz)
    for a, z in enumerate(zs):
        r = math.sqrt(1 - z * z)
        Fs = [oracle.cluster_free_energy(m, S, site, (r * math.cos(p), r * math.sin(p), z)) for p in phis]
        Fs = np.array(Fs)
        mx = (-Fs / m.T).max()
        logw[a] = mx + math.log(np.mean(np.exp(-Fs / m.T - mx)))
    w = np.exp(logw - logw.max())
    nbins = 8
    pb = w.reshape(nbins, nz // nbins).sum(axis=1)
    pb /= pb.sum()
    assert pb.max() / pb.min() > 3.0  # the weight is far from uniform
    steps, thin = 60000, 6
    trace, nacc = oracle.single_site_chain(m, S, site, 1000, steps)
    assert 0.05 < nacc / steps < 0.95
    z = trace[::thin, 2]
    counts, _ = np.histogram(z, bins=nbins, range=(-1, 1))
    expect = pb * z.size
    chi2 = float(np.sum((counts - expect) ** 2 / expect))
    assert chi2 < 40.0, (chi2, counts, expect)


# --------------------------------------------------------------------------
# Structure factor (Eq. 2)
# --------------------------------------------------------------------------
def test_structure_factor_ferro_and_neel():
    L = 6
    fm = inputs.ferro_spins(L * L, (0.3, 0.4, 0.5))
    af = inputs.neel_spins(L, L)
    assert abs(oracle.structure_factor(L, L, fm, 0, 0) - 1.0) < 1e-13
    assert abs(oracle.structure_factor(L, L, fm, math.pi, math.pi)) < 1e-13
    assert abs(oracle.structure_factor(L, L, af, math.pi, math.pi) - 1.0) < 1e-13
    assert abs(oracle.structure_factor(L, L, af, 0, 0)) < 1e-13


def test_structure_factor_sum_rule():
    # sum_q S(q) over the N lattice momenta equals (1/N) sum_i |S_i|^2 = 1.
    Lx, Ly = 4, 3
    S = inputs.random_unit_spins(12, Lx * Ly)
    tot = sum(oracle.structure_factor(Lx, Ly, S, 2 * math.pi * a / Lx, 2 * math.pi * b / Ly)
              for a in range(Lx) for b in range(Ly))
    assert abs(tot - 1.0) < 1e-12


# --------------------------------------------------------------------------
# Marshalling of the oracle's problem struct
# --------------------------------------------------------------------------
def test_oracle_model_struct_matches_the_c_layout(tmp_path):
    # The oracle source is compiled into a probe that prints sizeof and every
    # offsetof of oracle_model; the ctypes mirror must agree field by field.
    import ctypes
    import subprocess
    fields = [f for f, _ in oracle._Model._fields_ if not f.startswith("pad")]
    src = tmp_path / "layout.c"
    body = "\n".join(f'    printf("{f} %zu\\n", offsetof(oracle_model, {f}));' for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "ptca_oracle.c"\n'
                   'int main(void) {\n    printf("size %zu\\n", sizeof(oracle_model));\n' + body + "\n    return 0;\n}\n")
    exe = tmp_path / "layout"
    oracle_dir = os.path.join(os.path.dirname(GOLDEN), "..", "oracle")
    subprocess.run(["gcc", "-std=c11", "-I", oracle_dir, "-o", str(exe), str(src), "-lm"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {ln.split()[0]: int(ln.split()[1]) for ln in out if ln.strip()}
    assert got["size"] == ctypes.sizeof(oracle._Model)
    for f in fields:
        assert got[f] == getattr(oracle._Model, f).offset, f
