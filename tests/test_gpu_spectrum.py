"""Full-system spectrum (Sec. VI): all 2N eigenvalues of the whole lattice's
one-body Hamiltonian for the current configuration, against the oracle's
dense matrix of a window that covers the whole lattice (L_c = L), for each
model, open and periodic edges, a cube, a periodic axis of extent 2, a
two-site chain, and an order (2048) where the reduction runs over many tiles.
FP64 contexts reduce in FP64; PTCA_MIXED contexts run the reduction's pass
in double-float (about 48 significant bits) and are held to the same bound."""
import numpy as np
import pytest
import torch

import oracle
import paper_1502_07028_gb300 as P
from paper_1502_07028_gb300 import _build
from tests import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    assert torch.cuda.is_available()
    P.lib()


def _spectrum(cfg, S):
    ctx = P.Context(cfg)
    ctx.set_spins(S)
    eig = torch.empty(2 * cfg.N, dtype=torch.float64, device="cuda")
    P.ptca_full_spectrum(ctx.h, eig)
    ctx.close()
    return eig.cpu().numpy()


def _reference(cfg, S):
    L = max(cfg.Lx, cfg.Ly, cfg.Lz)
    m = oracle.Model(Lx=cfg.Lx, Ly=cfg.Ly, Lz=cfg.Lz, Lc=L, t=cfg.t, JH=cfg.J_H, lattice_periodic=cfg.periodic,
                     schedule=oracle.SCHEDULE_BLOCK, model=cfg.model, U=cfg.U, lam=cfg.lam, K=cfg.K)
    H, _ = oracle.cluster_hamiltonian(m, S, 0)
    assert H.shape[0] == 2 * cfg.N
    return np.sort(np.linalg.eigvalsh(H)), oracle.eigvalsh(H)


@pytest.mark.parametrize("case", [
    dict(cfg=dict(Lx=8, Ly=8, L_c=4), fields="unit"),
    dict(cfg=dict(Lx=6, Ly=6, L_c=3, periodic=0, schedule=P.SCHEDULE_BLOCK), fields="unit"),
    dict(cfg=dict(Lx=4, Ly=4, Lz=4, L_c=2), fields="unit"),
    dict(cfg=dict(Lx=2, Ly=2, L_c=2), fields="unit"),
    dict(cfg=dict(Lx=6, Ly=6, L_c=3, model=P.MODEL_HUBBARD_MF, U=6.0), fields="free"),
    dict(cfg=dict(Lx=40, Ly=1, L_c=8, model=P.MODEL_HOLSTEIN, lam=1.3), fields="scalar"),
    dict(cfg=dict(Lx=2, Ly=1, L_c=2), fields="unit"),
    dict(cfg=dict(Lx=3, Ly=1, L_c=3, periodic=0), fields="unit"),
    dict(cfg=dict(Lx=10, Ly=7, L_c=3, periodic=0, schedule=P.SCHEDULE_BLOCK), fields="unit"),
])
@pytest.mark.parametrize("precision", [P.FP64, P.MIXED])
def test_full_spectrum_matches_the_oracle(case, precision):
    cfg = P.Config(**case["cfg"], precision=precision)
    if case["fields"] == "unit":
        S = inputs.random_unit_spins(100 + cfg.N, cfg.N)
    elif case["fields"] == "free":
        S = inputs.random_fields(101, cfg.N, 2.0)
    else:
        S = np.zeros((cfg.N, 3))
        S[:, 0] = inputs.rng(102).uniform(-1.5, 1.5, size=cfg.N)
    got = _spectrum(cfg, S)
    lapack, jacobi = _reference(cfg, S)
    scale = 8.0 + 6.0
    assert np.max(np.abs(got - lapack)) <= 1e-10 * scale
    assert np.max(np.abs(got - jacobi)) <= 1e-10 * scale


def test_full_spectrum_rejects_lattices_beyond_its_limit():
    ctx = P.Context(P.Config(Lx=130, Ly=130, L_c=2))
    eig = torch.empty(2, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PtcaError) as e:
        P.ptca_full_spectrum(ctx.h, eig)
    assert e.value.status == 1
    ctx.close()


@pytest.mark.parametrize("precision", [P.FP64, P.MIXED])
def test_full_spectrum_at_order_2048_matches_lapack(precision):
    # 32x32 torus (n = 2048): 32 x 32 tiles of the reduction pass in its first
    # steps; checked against LAPACK's eigvalsh of the oracle's dense matrix.
    cfg = P.Config(Lx=32, Ly=32, L_c=4, precision=precision)
    S = inputs.random_unit_spins(7, cfg.N)
    got = _spectrum(cfg, S)
    m = oracle.Model(Lx=32, Ly=32, Lc=32, schedule=oracle.SCHEDULE_BLOCK)
    H, _ = oracle.cluster_hamiltonian(m, S, 0)
    ref = np.sort(np.linalg.eigvalsh(H))
    assert np.all(np.diff(got) >= 0)
    assert np.max(np.abs(got - ref)) <= 1e-10 * 14.0
    # trace and Frobenius norm of the spectrum against the matrix
    assert abs(got.sum() - np.trace(H).real) <= 1e-9 * cfg.N
    assert abs(np.sum(got ** 2) - np.sum(np.abs(H) ** 2)) <= 1e-9 * np.sum(np.abs(H) ** 2)
