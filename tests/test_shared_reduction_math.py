"""The fact the shared reduction (launch configuration reduction =
PTCA_REDUCTION_SHARED) rests on, checked in plain numpy (FP64, no GPU).

H_new differs from H_old only in the update site's 2x2 on-site block (the
proposal changes one classical vector; the hopping of Sec. II.c does not
depend on it).  With that block first in the basis, a block Householder
reduction in 2-column panels that starts below it never reads it, so the
2x2 block-tridiagonal (bandwidth 2) forms of H_old and H_new differ only in
their leading block; Givens rotations (a bulge chase) then make each band
tridiagonal without changing its eigenvalues.  Here: random Hermitian
matrices and cluster Hamiltonians of the double-exchange model, against
numpy's eigvalsh."""
import numpy as np
import pytest

import oracle
from tests import inputs


def _band_below_leading_block(H):
    """Block Householder with 2-column panels below the leading 2x2 block."""
    A = H.astype(np.complex128).copy()
    n = A.shape[0]
    for j in range(0, n - 2, 2):
        r0 = j + 2
        X = A[r0:, j:j + 2].copy()
        m = X.shape[0]
        Q = np.eye(m, dtype=np.complex128)
        for c in range(min(2, m)):
            x = X[c:, c]
            s = np.linalg.norm(x)
            if s == 0.0:
                continue
            a = x[0]
            ph = a / abs(a) if abs(a) > 0 else 1.0
            v = x.copy()
            v[0] += ph * s
            Hc = np.eye(m - c, dtype=np.complex128) - 2.0 * np.outer(v, v.conj()) / np.vdot(v, v).real
            X[c:, :] = Hc @ X[c:, :]
            Qc = np.eye(m, dtype=np.complex128)
            Qc[c:, c:] = Hc
            Q = Q @ Qc
        A[r0:, r0:] = Q.conj().T @ A[r0:, r0:] @ Q
        A[r0:, j:j + 2] = X
        A[j:j + 2, r0:] = X.conj().T
    return A


def _chase_to_tridiagonal(B):
    """Givens rotations: annihilate (k+2, k) with plane (k+1, k+2) and chase
    the bulge at (p+3, p) with planes (p+2, p+3)."""
    A = B.copy()
    n = A.shape[0]
    for k in range(n - 2):
        p, col = k + 1, k
        while p + 1 < n:
            q = p + 1
            a, b = A[p, col], A[q, col]
            rho = np.hypot(abs(a), abs(b))
            if rho == 0.0:
                break
            c = abs(a) / rho
            s = (a / abs(a)) * np.conj(b) / rho if abs(a) > 0 else 1.0
            if abs(a) == 0:
                c = 0.0
            G = np.eye(n, dtype=np.complex128)
            G[p, p] = c
            G[p, q] = s
            G[q, p] = -np.conj(s)
            G[q, q] = c
            A = G @ A @ G.conj().T
            if p + 3 < n and abs(A[p + 3, p]) > 1e-300:
                col, p = p, p + 2
            else:
                break
    return A


def _check_pair(Ho, Hn):
    n = Ho.shape[0]
    assert np.max(np.abs((Hn - Ho)[2:, :])) == 0.0 and np.max(np.abs((Hn - Ho)[:, 2:])) == 0.0
    Bo = _band_below_leading_block(Ho)
    Bn = _band_below_leading_block(Hn)
    # bandwidth 2, and the two bands differ only in the leading 2x2 block
    outside = np.abs(np.tril(Bo, -3))
    assert outside.max() <= 1e-12 * max(1.0, np.abs(Ho).max())
    assert np.array_equal(Bo[2:, :], Bn[2:, :]) and np.array_equal(Bo[:, 2:], Bn[:, 2:])
    # the old band with the new leading block is the new band
    Bmix = Bo.copy()
    Bmix[:2, :2] = Hn[:2, :2]
    for H, B in ((Ho, Bo), (Hn, Bmix)):
        T = _chase_to_tridiagonal(B)
        assert np.abs(np.tril(T, -2)).max() <= 1e-12 * max(1.0, np.abs(H).max())
        assert np.max(np.abs(np.linalg.eigvalsh(T) - np.linalg.eigvalsh(H))) <= 1e-12 * n * max(1.0, np.abs(H).max())


@pytest.mark.parametrize("n", [4, 6, 10, 16])
def test_random_hermitian_pairs(n):
    rng = inputs.rng(300 + n)
    H = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = (H + H.conj().T) / 2
    E = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    Hn = H.copy()
    Hn[:2, :2] += (E + E.conj().T) / 2
    _check_pair(H, Hn)


@pytest.mark.parametrize("lat", [dict(Lx=8, Ly=8, Lc=4), dict(Lx=9, Ly=1, Lc=5)])
def test_cluster_hamiltonians_of_an_update_site(lat):
    # the block schedule's update site is window site 0 (basis vectors 0, 1)
    m = oracle.Model(Lx=lat["Lx"], Ly=lat["Ly"], Lc=lat["Lc"], JH=8.0, schedule=oracle.SCHEDULE_BLOCK, seed=1)
    S = inputs.random_unit_spins(11, m.Lx * m.Ly)
    site = 3
    s_new = inputs.random_unit_spins(12, 1)[0]
    Ho = oracle.cluster_hamiltonian(m, S, site)[0]
    Hn = oracle.cluster_hamiltonian(m, S, site, s_new)[0]
    _check_pair(Ho, Hn)
