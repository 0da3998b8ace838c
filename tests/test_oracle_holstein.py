"""Pins of the oracle's adiabatic Holstein model (Sec. VII.b): one classical
distortion x_i per site, one-body term lambda x_i n_i (spin-independent, so
the cluster matrix is real and block diagonal in spin), and the classical
energy K/2 x_i^2 - lambda x_i + mu of every window site.  What the
mathematics fixes: the chain's tight-binding spectrum (lambda = 0), a uniform
shift (uniform x), decoupled sites (t = 0), the distributions of the initial
distortions and of the proposal, and the Boltzmann weight of one site."""
import math

import numpy as np
import pytest

import oracle
from tests import inputs


def _hol(**kw):
    base = dict(Lx=32, Ly=1, Lc=8, t=1.0, lam=1.5, K=1.0, mu=0.0, T=0.1, m_step=0.4,
                model=oracle.MODEL_HOLSTEIN, schedule=oracle.SCHEDULE_BLOCK)
    base.update(kw)
    return oracle.Model(**base)


def _f(eps, mu, T):
    x = -(eps - mu) / T
    return -T * ((x if x > 0 else 0.0) + math.log1p(math.exp(-abs(x))))


def _fields(seed, N, r):
    S = np.zeros((N, 3))
    S[:, 0] = inputs.rng(seed).uniform(-r, r, size=N)
    return S


@pytest.mark.parametrize("Lc", [3, 5, 8])
def test_zero_coupling_gives_the_chain_spectrum_twice(Lc):
    m = _hol(lam=0.0, Lc=Lc)
    e = oracle.eigvalsh(oracle.cluster_hamiltonian(m, _fields(1, m.N, 1.0), 5)[0])
    k = np.sort([-2.0 * math.cos(2 * math.pi * a / Lc) for a in range(Lc)])
    assert np.max(np.abs(e - np.sort(np.concatenate([k, k])))) < 1e-12


def test_uniform_distortion_shifts_the_open_chain_spectrum():
    m = _hol(Lx=20, Lc=6, lattice_periodic=0, cluster_periodic=0, lam=0.7, t=1.3)
    S = np.zeros((m.N, 3))
    S[:, 0] = -0.8
    e = oracle.eigvalsh(oracle.cluster_hamiltonian(m, S, 10)[0])
    k = np.sort([-2.6 * math.cos(math.pi * a / 7) for a in range(1, 7)])
    assert np.max(np.abs(e - (np.sort(np.concatenate([k, k])) - 0.56))) < 1e-12


def test_cluster_matrix_is_real_and_spin_block_diagonal():
    m = _hol()
    H = oracle.cluster_hamiltonian(m, _fields(2, m.N, 1.5), 11)[0]
    assert np.max(np.abs(H.imag)) == 0.0
    assert np.max(np.abs(H[0::2, 1::2])) == 0.0
    assert np.max(np.abs(H[0::2, 0::2] - H[1::2, 1::2])) == 0.0


def test_zero_hopping_free_energy_closed_form():
    m = _hol(t=0.0, lam=1.2, K=0.8, mu=0.3, T=0.25, Lc=5)
    S = _fields(3, m.N, 1.5)
    s_new = np.array([0.9, 0.0, 0.0])
    for site in (0, 17, 31):
        for sn in (None, s_new):
            F = 0.0
            for g in range(m.N):
                if not oracle.in_window(m, site, g):
                    continue
                x = float(sn[0]) if (sn is not None and g == site) else float(S[g, 0])
                F += 2 * _f(1.2 * x, 0.3, 0.25) + 0.4 * x * x - 1.2 * x + 0.3
            got = oracle.cluster_free_energy(m, S, site, sn)
            assert abs(got - F) < 1e-11 * max(1.0, abs(F))


def test_initial_distortions_and_proposal_are_uniform():
    m = _hol(Lx=4000, seed=9)
    S = oracle.init_spins(m)
    x = S[:, 0]
    assert np.all(S[:, 1:] == 0.0) and np.all(np.abs(x) < 1.0)
    n = x.size
    assert abs(x.mean()) < 4 * math.sqrt(1 / 3 / n)
    assert abs((x ** 2).mean() - 1 / 3) < 4 * math.sqrt((1 / 5 - 1 / 9) / n)
    d = np.array([oracle.propose(m, sw, site, np.array([0.3, 0.0, 0.0]))[0] - 0.3
                  for sw in range(10) for site in range(2000)])
    n = d.size
    assert np.all(np.abs(d) <= 0.4 + 1e-15)
    assert abs(d.mean()) < 4 * 0.4 / math.sqrt(3 * n)
    assert abs((d ** 2).mean() - 0.16 / 3) < 4 * 0.16 * math.sqrt((1 / 5 - 1 / 9) / n)


def test_single_site_chain_samples_the_boltzmann_weight():
    # t = 0: p(x) ~ exp(-g(x)/T), g(x) = 2 f(lambda x) + K/2 x^2 - lambda x,
    # a double well with minima near x = -+lambda/K (particle-hole symmetry).
    lam, K, mu, T = 1.5, 1.0, 0.0, 0.3
    m = _hol(Lx=8, Lc=2, t=0.0, lam=lam, K=K, mu=mu, T=T, m_step=0.8, seed=4)
    S = np.zeros((m.N, 3))

    def g(x):
        return 2 * _f(lam * x, mu, T) + 0.5 * K * x * x - lam * x

    edges = np.linspace(-5.0, 5.0, 21)
    xx = np.linspace(-5.0, 5.0, 20001)
    gm = min(g(x) for x in xx[::40])
    dens = np.array([math.exp(-(g(x) - gm) / T) for x in xx])
    pb = np.array([np.trapezoid(dens[(xx >= a) & (xx <= b)], xx[(xx >= a) & (xx <= b)])
                   for a, b in zip(edges[:-1], edges[1:])])
    pb /= np.trapezoid(dens, xx)
    steps, thin = 60000, 6
    trace, nacc = oracle.single_site_chain(m, S, 3, 500, steps)
    assert 0.1 < nacc / steps < 0.95
    x = trace[::thin, 0]
    assert x.min() > -5.0 and x.max() < 5.0
    counts, _ = np.histogram(x, bins=edges)
    expect = pb * x.size
    keep = expect > 5
    chi2 = float(np.sum((counts[keep] - expect[keep]) ** 2 / expect[keep]))
    assert chi2 < 45.0, (chi2, counts, expect)


def _binned(x, nb=16):
    b = np.asarray(x)[: len(x) // nb * nb].reshape(nb, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nb)


def test_corner_and_central_update_sites_give_the_same_order_and_energy():
    # Sec. VII.b: the 'corner' and the 'central' choice of update site give
    # the same charge order N(pi) and energy.  Both chains start from the
    # charge-density wave (from random distortions the domains of either
    # scheme coarsen slowly) on a 32-site ring with N_c = 8; the means over
    # 800 sweeps, with errors from 16 bins, must agree within 2 sigma.
    N, T, sweeps, burn = 32, 0.1, 900, 100
    stats = []
    for central in (False, True):
        if central:
            m = _hol(Lx=N, Lc=8, T=T, seed=5, schedule=oracle.SCHEDULE_TILED, stride=8, ox=4)
        else:
            m = _hol(Lx=N, Lc=8, T=T, seed=5, schedule=oracle.SCHEDULE_BLOCK, ox=0)
        S = np.zeros((N, 3))
        S[:, 0] = 1.2 * (-1.0) ** np.arange(N)
        n_pi, f_site = [], []
        for sw in range(sweeps):
            S, rec = oracle.sweep(m, S, sw)
            if sw >= burn:
                n_pi.append(oracle.structure_factor(N, 1, S, math.pi, 0.0))
                f_site.append(np.mean(np.where(rec.accepted == 1, rec.F_new, rec.F_old)) / 8)
        stats.append((_binned(n_pi), _binned(f_site)))
    (nc, fc), (nm, fm) = stats
    assert nc[0] > 1.0 and nm[0] > 1.0           # ordered at T = 0.1
    assert abs(nc[0] - nm[0]) < 2 * math.hypot(nc[1], nm[1]), (nc, nm)
    assert abs(fc[0] - fm[0]) < 2 * math.hypot(fc[1], fm[1]), (fc, fm)
