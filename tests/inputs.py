"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module only draws numbers and lays out configurations; it holds none of
the method's arithmetic (no Hamiltonian, eigenvalue, free-energy or Metropolis
code).  Both sides of every parity test read the same arrays from here.
"""
import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def random_unit_spins(seed: int, N: int) -> np.ndarray:
    """N classical unit vectors, isotropic (normalised Gaussian triples)."""
    g = rng(seed).normal(size=(N, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def ferro_spins(N: int, direction) -> np.ndarray:
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return np.tile(d, (N, 1))


def neel_spins(Lx: int, Ly: int, direction=(0.0, 0.0, 1.0)) -> np.ndarray:
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    x, y = np.meshgrid(np.arange(Lx), np.arange(Ly))
    sign = np.where(((x + y) % 2).ravel() == 0, 1.0, -1.0)
    return sign[:, None] * d[None, :]


def random_rotation(seed: int) -> np.ndarray:
    """Uniform random 3x3 rotation (QR of a Gaussian matrix, det +1)."""
    q, r = np.linalg.qr(rng(seed).normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def random_hermitian(seed: int, n: int, scale: float = 1.0) -> np.ndarray:
    g = rng(seed)
    a = g.normal(size=(n, n)) + 1j * g.normal(size=(n, n))
    return scale * (a + a.conj().T) / 2.0


def random_sites(seed: int, N: int, m: int) -> np.ndarray:
    return rng(seed).choice(N, size=m, replace=False).astype(np.int32)


def random_fields(seed: int, N: int, rmax: float) -> np.ndarray:
    """N classical vectors with isotropic directions and lengths uniform in
    [0, rmax] (mean-field magnetisations of any length)."""
    g = rng(seed)
    d = g.normal(size=(N, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * g.uniform(0.0, rmax, size=(N, 1))
