"""Pins of the oracle's Hubbard mean-field model (Eq. 1 with <n_i> = 1).

Each cluster site carries the on-site block (U/2)(1 - m_i . sigma) with a
classical vector m_i of any length, and the cluster free energy adds the
classical energy (U/4)(m_i^2 - 1) of every window site.  The pins use what the
mathematics fixes: tight-binding spectra shifted by U/2 (m = 0), the
ferromagnetic closed form with splitting U|m| (uniform m), the exact relation
to the double-exchange matrix for unit fields, decoupled sites (t = 0), the
distribution of the ball proposal, and the Boltzmann weight sampled by a
single-site chain."""
import math

import numpy as np
import pytest

import oracle
from tests import inputs


def _tb_fm_periodic(Lc, t, split):
    k = [-2 * t * (math.cos(2 * math.pi * a / Lc) + math.cos(2 * math.pi * b / Lc))
         for a in range(Lc) for b in range(Lc)]
    return np.sort(np.array([e + s for e in k for s in (-split, split)]))


def _tb_fm_open(ex, ey, t, split):
    kx = [-2 * t * math.cos(math.pi * a / (ex + 1)) for a in range(1, ex + 1)]
    ky = [-2 * t * math.cos(math.pi * b / (ey + 1)) for b in range(1, ey + 1)]
    return np.sort(np.array([x + y + s for x in kx for y in ky for s in (-split, split)]))


def _hub(**kw):
    base = dict(Lx=8, Ly=8, Lc=4, t=1.0, U=8.0, mu=4.0, T=0.1, model=oracle.MODEL_HUBBARD_MF, m_step=0.5)
    base.update(kw)
    return oracle.Model(**base)


def _f(eps, mu, T):
    x = -(eps - mu) / T
    return -T * ((x if x > 0 else 0.0) + math.log1p(math.exp(-abs(x))))


@pytest.mark.parametrize("Lc", [2, 3, 4])
def test_zero_field_is_tight_binding_shifted_by_half_U(Lc):
    m = _hub(Lc=Lc, U=6.0)
    S = np.zeros((m.N, 3))
    e = oracle.eigvalsh(oracle.cluster_hamiltonian(m, S, 9)[0])
    assert np.max(np.abs(e - (_tb_fm_periodic(Lc, 1.0, 0.0) + 3.0))) < 1e-12


@pytest.mark.parametrize("c", [0.3, 1.0, 1.7])
def test_uniform_field_splits_by_U_times_length(c):
    # m_i = c d for all i: eps = eps_TB + U/2 -+ (U/2) c.
    m = _hub(U=5.0, t=1.2)
    S = inputs.ferro_spins(m.N, (0.3, -0.4, 0.8)) * c
    e = oracle.eigvalsh(oracle.cluster_hamiltonian(m, S, 17)[0])
    assert np.max(np.abs(e - (_tb_fm_periodic(4, 1.2, 2.5 * c) + 2.5))) < 1e-12
    mo = _hub(U=5.0, t=1.2, cluster_periodic=0)
    e = oracle.eigvalsh(oracle.cluster_hamiltonian(mo, S, 17)[0])
    assert np.max(np.abs(e - (_tb_fm_open(4, 4, 1.2, 2.5 * c) + 2.5))) < 1e-12


def test_unit_fields_give_the_double_exchange_matrix_plus_half_U():
    # |m_i| = 1: H_Hubb-MF(U) = H_DE(J_H = U/2) + (U/2) 1, element by element.
    S = inputs.random_unit_spins(4, 64)
    mh = _hub(U=7.0)
    md = oracle.Model(Lx=8, Ly=8, Lc=4, t=1.0, JH=3.5)
    for site in (0, 27, 63):
        Hh = oracle.cluster_hamiltonian(mh, S, site)[0]
        Hd = oracle.cluster_hamiltonian(md, S, site)[0]
        assert np.max(np.abs(Hh - Hd - 3.5 * np.eye(Hh.shape[0]))) < 1e-14


def test_zero_hopping_free_energy_closed_form():
    # t = 0: every site is a two-level system U/2 -+ (U/2)|m_i|; the cluster
    # free energy adds (U/4)(|m_i|^2 - 1) for every window site.
    m = _hub(t=0.0, U=6.0, mu=2.5, T=0.3, Lc=3)
    S = inputs.random_fields(8, m.N, 1.8)
    s_new = np.array([0.4, -1.1, 0.2])
    for site in (0, 30, 63):
        for sn in (None, s_new):
            win = [g for g in range(m.N) if oracle.in_window(m, site, g)]
            F = 0.0
            for g in win:
                v = sn if (sn is not None and g == site) else S[g]
                r = float(np.linalg.norm(v))
                F += _f(3.0 - 3.0 * r, 2.5, 0.3) + _f(3.0 + 3.0 * r, 2.5, 0.3) + 1.5 * (r * r - 1.0)
            got = oracle.cluster_free_energy(m, S, site, sn)
            assert abs(got - F) < 1e-11 * max(1.0, abs(F)), (site, got, F)


def test_classical_energy_enters_dF_through_the_update_site_only():
    # F_total - F_one-body is the window's classical energy; between old and
    # new states it changes by (U/4)(|m_new|^2 - |m_old|^2).
    m = _hub(U=8.0, mu=4.0, T=0.2)
    S = inputs.random_fields(9, m.N, 1.5)
    site = 36
    s_new = np.array([0.9, 0.2, -0.6])
    parts = []
    for sn in (None, s_new):
        H = oracle.cluster_hamiltonian(m, S, site, sn)[0]
        fb = oracle.free_energy(oracle.eigvalsh(H), m.mu, m.T)
        parts.append(oracle.cluster_free_energy(m, S, site, sn) - fb)
    win = [g for g in range(m.N) if oracle.in_window(m, site, g)]
    expect_old = sum(2.0 * (float(S[g] @ S[g]) - 1.0) for g in win)
    assert abs(parts[0] - expect_old) < 1e-12
    assert abs((parts[1] - parts[0]) - 2.0 * (float(s_new @ s_new) - float(S[site] @ S[site]))) < 1e-12


def test_ball_proposal_is_uniform_in_the_ball_around_the_old_field():
    m = _hub(m_step=0.7, seed=13)
    s_old = np.array([0.2, -0.9, 0.4])
    d = np.array([oracle.propose(m, sw, site, s_old) - s_old for sw in range(40) for site in range(500)])
    r = np.linalg.norm(d, axis=1)
    n = len(d)
    assert r.max() <= 0.7 + 1e-12
    # E[d] = 0, E|d|^2 = 3/5 step^2, P(|d| <= x step) = x^3, isotropic directions.
    assert np.all(np.abs(d.mean(axis=0)) < 4 * 0.7 / math.sqrt(5 * n))
    var_r2 = 0.7 ** 4 * (3 / 7 - 9 / 25)
    assert abs((r ** 2).mean() - 0.6 * 0.49) < 4 * math.sqrt(var_r2 / n)
    for x in (0.3, 0.5, 0.8):
        p = x ** 3
        assert abs((r <= x * 0.7).mean() - p) < 4 * math.sqrt(p * (1 - p) / n)
    u = d / r[:, None]
    assert np.all(np.abs(u.mean(axis=0)) < 4 / math.sqrt(3 * n))


def test_single_site_chain_samples_the_radial_boltzmann_weight():
    # t = 0 decouples the sites, so the chain of one field samples
    # p(m) ~ exp(-g(|m|)/T) d^3m with g(r) = f(U/2 - Ur/2) + f(U/2 + Ur/2)
    # + (U/4)(r^2 - 1): radial density ~ r^2 exp(-g(r)/T), peaked near the
    # mean-field moment r = 1 at mu = U/2.
    U, T, mu = 4.0, 0.5, 2.0
    m = _hub(Lx=4, Ly=4, Lc=2, t=0.0, U=U, mu=mu, T=T, m_step=0.6, seed=5)
    S = np.zeros((m.N, 3))
    S[:, 2] = 1.0

    def g(r):
        return _f(U / 2 - U * r / 2, mu, T) + _f(U / 2 + U * r / 2, mu, T) + U / 4 * (r * r - 1)

    edges = np.linspace(0.0, 4.0, 11)
    rr = np.linspace(0.0, 4.0, 8001)
    dens = np.array([r * r * math.exp(-(g(r) - g(1.0)) / T) for r in rr])
    pb = np.array([np.trapezoid(dens[(rr >= a) & (rr <= b)], rr[(rr >= a) & (rr <= b)])
                   for a, b in zip(edges[:-1], edges[1:])])
    tail = np.trapezoid(dens, rr)
    pb /= tail
    steps, thin = 60000, 6
    trace, nacc = oracle.single_site_chain(m, S, 5, 2000, steps)
    assert 0.1 < nacc / steps < 0.95
    r = np.linalg.norm(trace[::thin], axis=1)
    assert r.max() < 4.0
    counts, _ = np.histogram(r, bins=edges)
    expect = pb * r.size
    keep = expect > 5
    chi2 = float(np.sum((counts[keep] - expect[keep]) ** 2 / expect[keep]))
    assert chi2 < 40.0, (chi2, counts, expect)
